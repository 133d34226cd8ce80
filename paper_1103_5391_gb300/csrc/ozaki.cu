// Mixed-precision superblock products on the tcgen05 tensor cores (Sec. IV, Hamiltonian connections).
//
// Each complex product C (+)= A op(B) of a task is carried out exactly in integer slices
// (Ozaki-style splitting), so the only approximation is the truncation of the operands:
//   real embedding     A' = [Re A | Im A]  (M x 2K),   B'^T rows = [Re b_j | -Im b_j], [Im b_j | Re b_j];
//   common exponents   E_i over row i of A' (all segments of the task), F_j over column j of B';
//   fixed point        a = v 2^{-E} in (-1, 1),  N = round(a 2^{7S})  (integer arithmetic only);
//   balanced digits    N = sum_s d_s 2^{7(S-s)},  |d_1| <= 128, |d_s| <= 64  (exact in bf16);
//   slice products     X_g = sum_{s+t=g} A^(s) B^(t)^T for g = 2..S+1, one TMEM accumulator per g,
//                      exact in the FP32 accumulator as long as a readout block spans <= 512 real K;
//   recombination      C' = sum_g X_g 2^{7(S+1-g)} 2^{E_i + F_j - 7(S+1)} in int64, one conversion.
// The error is about 2^{-7S} of max|A'_i| max|B'_j| per entry (S = ozaki_slices).
//
// Operands are pre-sliced into bf16 panels in global memory ("slice planes": plane s holds digit s of
// every row, K-major, rows of kpad elements) and staged into shared memory by TMA (2-D tensor maps,
// 128-byte swizzle); one elected thread issues tcgen05.mma (kind::f16, bf16 x bf16 -> f32, M = 128,
// N = 2 n_t <= 64) into TMEM, the four warps read the accumulators back with tcgen05.ld.
// Static operands (operator blocks with the term coefficients and fermion signs folded in) are
// sliced once per plan; the wave function and the stage-1 intermediates are sliced per product.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "internal.h"

namespace tdmrg {
namespace {

constexpr int KCH = 64;         // K per TMA box / smem stage (64 bf16 = 128 B rows)
constexpr int TM = 128;         // MMA M
constexpr int TNC = 32;         // complex output columns per tile (MMA N = 2 * n_t <= 64)
constexpr int ABOX = TM * KCH * 2;         // bytes of one A slice box (16 KB)
constexpr int BBOX = 2 * TNC * KCH * 2;    // bytes of one B slice box (8 KB)
constexpr int kReadoutChunks = 8;          // 8 x 64 = 512 real K per exact accumulation block
constexpr long kWaitLimit = 1L << 26;      // bounded mbarrier polls

// ------------------------------------------------------------------------------ slicing
__device__ __forceinline__ int biased_exp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF); }

// round(v * 2^{S7 - E}) with integer arithmetic (|v| < 2^E); zero and subnormals give 0
__device__ __forceinline__ long long fixed_point(double v, int E, int S7) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0) return 0;
    const long long m = (long long)((b & ((1ull << 52) - 1)) | (1ull << 52));
    const int sh = (ex - 1075) + S7 - E;
    long long r;
    if (sh >= 0) r = m << sh;
    else if (sh < -62) r = 0;
    else r = (m + (1ll << (-sh - 1))) >> (-sh);
    return (b >> 63) ? -r : r;
}

template <int S>
__device__ __forceinline__ void digits(long long N, int* d) {
#pragma unroll
    for (int s = 1; s < S; ++s) {
        const int w = 7 * (S - s);
        const long long q = (N + (1ll << (w - 1))) >> w;
        N -= q << w;
        d[s - 1] = (int)q;
    }
    d[S - 1] = (int)N;
}

__device__ __forceinline__ double2 scaled(double2 v, cplx s) {
    return make_double2(s.x * v.x - s.y * v.y, s.x * v.y + s.y * v.x);
}

// For S <= 4 the fixed-point value fits 32 bits (|N| <= 2^28), so the rounding and the digits run in
// 32-bit integer arithmetic: with k = -sh >= 25, (m + 2^{k-1}) >> k = ((m >> (k - 1)) + 1) >> 1, whose
// operand is below 2^29.  Same values as fixed_point + digits.
template <int S>
__device__ __forceinline__ void slice_digits(double v, int E, int* d) {
    if constexpr (7 * S <= 28) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        const int ex = (int)((b >> 52) & 0x7FF);
        int N = 0;
        if (ex != 0) {
            const int k = E - (ex - 1075) - 7 * S;   // >= 25 as |v| < 2^E
            if (k <= 62) {
                const unsigned long long m = (b & ((1ull << 52) - 1)) | (1ull << 52);
                N = (int)(((unsigned)(m >> (k - 1)) + 1u) >> 1);
                if (b >> 63) N = -N;
            }
        }
#pragma unroll
        for (int s = 1; s < S; ++s) {
            const int w = 7 * (S - s);
            const int q = (N + (1 << (w - 1))) >> w;
            N -= q << w;
            d[s - 1] = q;
        }
        d[S - 1] = N;
    } else {
        digits<S>(fixed_point(v, E, 7 * S), d);
    }
}

// One CTA of kSliceCT threads per vector (row of A' or complex column of B'); two passes over the task's
// segments (exponent, then digits).  The segments are flattened into one element index (their views
// cached in shared memory, kSegCache at a time) and each thread loads kSliceCU elements per batch, so a
// vector costs a few memory latencies, its elements spread over four warps; a vector of at most
// kSliceCT kSliceCU elements keeps its values in registers between the passes.
constexpr int kSliceCT = 128;
constexpr int kSliceCU = 4;
constexpr int kSegCache = 16;

struct SegView {          // element k of the vector at base[k * sk], conjugated and scaled as asked
    const double2* base;
    int64_t sk;
    double2 scale;
    int conj;
};

__device__ __forceinline__ double2 view_load(const SegView& w, int k, bool use_scale) {
    double2 x = w.base[(int64_t)k * w.sk];
    if (w.conj) x.y = -x.y;
    if (use_scale) x = scaled(x, w.scale);
    return x;
}

template <int S>
__global__ void __launch_bounds__(kSliceCT) k_slice(OzSliceArgs sa, GemmArgs g, const int* skip_flag, int skip_step) {
    pdl_enter();
    if (skip_flag != nullptr && skip_step >= *skip_flag) return;
    const int gv = blockIdx.x;   // the vector; block-uniform
    if (gv >= sa.nvec_total) return;
    const int tid = threadIdx.x, lane = tid & 31, wi = tid >> 5;
    const OzSliceJob job = sa.jobs[sa.vjob[gv]];
    const int v = gv - job.vec_prefix;
    __shared__ SegView sv[kSegCache];
    __shared__ int spre[kSegCache + 1];
    __shared__ int red[kSliceCT / 32];
    const int nseg = job.seg_end - job.seg_begin;
    const bool use_scale = job.use_scale != 0;
    // views of segments [w0, w0 + nw) for this vector and the prefix offsets of their K (warp 0, one scan)
    auto build = [&](int w0, int nw, bool again) {
        if (again) __syncthreads();   // the previous window's views are no longer read
        if (wi == 0) {
            int k = 0;
            if (lane < nw) {
                const Seg sg = sa.segs[job.seg_begin + w0 + lane];
                SegView w;
                w.scale = sg.scale;
                if (sg.dcoef >= 0 && g.dcoef != nullptr) w.scale = scaled(g.dcoef[sg.dcoef], sg.scale);   // run-time coefficient
                w.conj = 0;
                if (job.role == 0) {
                    w.base = g.bufs[sg.a_buf] + sg.a_off + (int64_t)v * sg.lda;
                    w.sk = 1;
                } else {
                    const cplx* B = g.bufs[sg.b_buf] + sg.b_off;
                    if (sg.opb == OPB_N) { w.base = B + v; w.sk = sg.ldb; }
                    else { w.base = B + (int64_t)v * sg.ldb; w.sk = 1; w.conj = sg.opb == OPB_C; }
                }
                sv[lane] = w;
                k = sg.K;
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {   // inclusive prefix sum over the lanes
                const int t = __shfl_up_sync(0xffffffffu, k, o);
                if (lane >= o) k += t;
            }
            if (lane < nw) spre[lane + 1] = k;
            if (lane == 0) spre[0] = 0;
        }
        __syncthreads();
        return spre[nw];
    };
    auto seg_of = [&](int e, int nw) {
        int sgi = 0;
        while (sgi + 1 < nw && e >= spre[sgi + 1]) ++sgi;
        return sgi;
    };
    const bool one_window = nseg <= kSegCache;
    double2 xr[kSliceCU];
    int emax = 0, kw_first = 0;
    for (int w0 = 0; w0 < nseg; w0 += kSegCache) {   // pass 1: largest exponent
        const int nw = min(kSegCache, nseg - w0);
        const int kw = build(w0, nw, w0 > 0);
        if (w0 == 0) kw_first = kw;
        for (int e0 = 0; e0 < kw; e0 += kSliceCT * kSliceCU) {
            double2 x[kSliceCU];
#pragma unroll
            for (int u = 0; u < kSliceCU; ++u) {
                const int e = e0 + tid + kSliceCT * u;
                x[u] = make_double2(0.0, 0.0);
                if (e < kw) {
                    const int sgi = seg_of(e, nw);
                    x[u] = view_load(sv[sgi], e - spre[sgi], use_scale);
                }
            }
#pragma unroll
            for (int u = 0; u < kSliceCU; ++u) {
                emax = max(emax, max(biased_exp(x[u].x), biased_exp(x[u].y)));
                if (w0 == 0 && e0 == 0) xr[u] = x[u];
            }
        }
    }
    const bool cached = one_window && kw_first <= kSliceCT * kSliceCU;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    if (lane == 0) red[wi] = emax;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSliceCT / 32; ++k) emax = max(emax, red[k]);
    const int E = emax == 0 ? 0 : emax - 1023 + 1;   // every |value| < 2^E
    int r_re, r_im;                                   // destination panel rows
    if (job.role == 0) {
        r_re = r_im = job.row0 + v;
    } else {
        // column c of a column tile: rows 2c (Re) and 2c + 1 (Im) of the tile's 2 n_t rows, so the two
        // accumulator columns of one complex output are adjacent (one 16-byte store in the epilogue)
        const int nt = v / TNC, c = v % TNC;
        r_re = job.row0 + 2 * TNC * nt + 2 * c;
        r_im = r_re + 1;
    }
    if (tid == 0) sa.exps[job.exp0 + v] = E;
    const int64_t plane = (int64_t)sa.rows * sa.kpad;
    __nv_bfloat16* const row_re = sa.panel + (int64_t)r_re * sa.kpad;   // plane 0 rows; plane t at + t plane
    __nv_bfloat16* const row_im = sa.panel + (int64_t)r_im * sa.kpad;
    const bool role0 = job.role == 0;
    const int q = job.ktot;   // the imaginary half of a row starts at ktot
    int kbase = 0;
    for (int w0 = 0; w0 < nseg; w0 += kSegCache) {   // pass 2: digits
        const int nw = min(kSegCache, nseg - w0);
        const int kw = one_window ? kw_first : build(w0, nw, true);
        for (int e0 = 0; e0 < kw; e0 += kSliceCT * kSliceCU) {
#pragma unroll
            for (int u = 0; u < kSliceCU; ++u) {
                const int e = e0 + tid + kSliceCT * u;
                if (e < kw) {
                    double2 x;
                    if (cached) {
                        x = xr[u];
                    } else {
                        const int sgi = seg_of(e, nw);
                        x = view_load(sv[sgi], e - spre[sgi], use_scale);
                    }
                    int dr[S], di[S];
                    slice_digits<S>(x.x, E, dr);
                    slice_digits<S>(x.y, E, di);
                    __nv_bfloat16* pr = row_re + kbase + e;
                    __nv_bfloat16* pi = row_im + kbase + e;
#pragma unroll
                    for (int t = 0; t < S; ++t) {
                        if (role0) {
                            pr[t * plane] = __float2bfloat16_rn((float)dr[t]);
                            pr[t * plane + q] = __float2bfloat16_rn((float)di[t]);
                        } else {
                            pr[t * plane] = __float2bfloat16_rn((float)dr[t]);
                            pr[t * plane + q] = __float2bfloat16_rn((float)(-di[t]));
                            pi[t * plane] = __float2bfloat16_rn((float)di[t]);
                            pi[t * plane + q] = __float2bfloat16_rn((float)dr[t]);
                        }
                    }
                }
            }
        }
        kbase += kw;
    }
}

// ------------------------------------------------------------------------------ tcgen05 GEMM
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// a * 2^e as a double, rounded to nearest even, built with integer operations only (the FP64 units
// of this GPU are ~60x slower than its integer ones); results below the normal range flush to zero
__device__ __forceinline__ double scaled_int(long long a, int e) {
    if (a == 0) return 0.0;
    const unsigned long long sign = a < 0 ? (1ull << 63) : 0ull;
    unsigned long long u = a < 0 ? (unsigned long long)(-a) : (unsigned long long)a;
    const int lz = __clzll(u);
    u <<= lz;                                             // leading one at bit 63
    unsigned long long mant = u >> 11;                    // 53 bits
    const unsigned long long rest = u & 0x7FFull;
    if (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ++mant;
    int ex = 63 - lz + e;
    if (mant >> 53) { mant >>= 1; ++ex; }
    const int biased = ex + 1023;
    if (biased <= 0) return 0.0;
    return __longlong_as_double((long long)(sign | ((unsigned long long)biased << 52) | (mant & ((1ull << 52) - 1))));
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 :: "r"(dst), "l"(map), "r"(x), "r"(y), "r"(bar) : "memory");
}

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

template <int S>
__global__ void __launch_bounds__(128) k_ozaki_gemm(const __grid_constant__ CUtensorMap mapA,
                                                     const __grid_constant__ CUtensorMap mapB, OzGemmArgs oa, GemmArgs g,
                                                     const int* skip_flag, int skip_step) {
    pdl_enter();
    if (skip_flag != nullptr && skip_step >= *skip_flag) return;
    constexpr int NCOLS = (S * 64 <= 256) ? 256 : 512;   // TMEM columns: one 64-column accumulator per g
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = smem;                 // S boxes of 16 KB
    unsigned char* sB = smem + S * ABOX;      // S boxes of 8 KB
    __shared__ __align__(8) uint64_t bar_tma, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const OzTile tile = oa.tiles[blockIdx.x];
    const OzTask task = oa.tasks[tile.task];
    const int nrem = task.N - tile.n0;
    const int nval = nrem < TNC ? nrem : TNC;          // valid complex columns of this tile
    const int n_t = (nval + 7) & ~7;                    // MMA N = 2 n_t (multiple of 16)
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((2 * n_t) >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
    if (tid == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar_tma)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tmem_base)), "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    long long acc[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) acc[j] = 0;
    const int ya = task.arow0 + tile.m0;
    const int yb = task.brow0 + 2 * tile.n0;   // the tile's rows start 2 * TNC rows per full tile
    uint32_t phase = 0;
    for (int c = 0; c < task.kchunks; ++c) {
        if (tid == 0 && !failed) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(&bar_tma)), "r"(S * (ABOX + BBOX)) : "memory");
#pragma unroll
            for (int s = 0; s < S; ++s) {
                tma_load(smem_u32(sA + s * ABOX), &mapA, c * KCH, s * oa.rowsA + ya, smem_u32(&bar_tma));
                tma_load(smem_u32(sB + s * BBOX), &mapB, c * KCH, s * oa.rowsB + yb, smem_u32(&bar_tma));
            }
        }
        if (!mbar_wait(smem_u32(&bar_tma), phase)) failed = 1;
        __syncthreads();
        const bool first_in_block = (c % kReadoutChunks) == 0;
        if (tid == 0 && !failed) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int ks = 0; ks < KCH / 16; ++ks) {
#pragma unroll
                for (int gg = 2; gg <= S + 1; ++gg) {
                    const int s_lo = gg - S > 1 ? gg - S : 1, s_hi = gg - 1 < S ? gg - 1 : S;
#pragma unroll
                    for (int s = s_lo; s <= s_hi; ++s) {
                        const int t = gg - s;
                        const uint64_t da = desc_sw128(smem_u32(sA + (s - 1) * ABOX) + ks * 32);
                        const uint64_t db = desc_sw128(smem_u32(sB + (t - 1) * BBOX) + ks * 32);
                        const uint32_t accum = (first_in_block && ks == 0 && s == s_lo) ? 0u : 1u;
                        umma(tmem + (uint32_t)((gg - 2) * 64), da, db, idesc, accum);
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_u32(&bar_mma)) : "memory");
        }
        if (!mbar_wait(smem_u32(&bar_mma), phase)) failed = 1;   // smem stage free, accumulators complete
        __syncthreads();
        phase ^= 1;
        if (failed) break;
        if ((c % kReadoutChunks) == kReadoutChunks - 1 || c == task.kchunks - 1) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int gg = 2; gg <= S + 1; ++gg) {
                const int shift = 7 * (S + 1 - gg);
                uint32_t r[4][16];
#pragma unroll
                for (int cb = 0; cb < 4; ++cb)   // all loads of the group in flight, one wait
                    if (cb * 16 < 2 * n_t)
                        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)((gg - 2) * 64 + cb * 16), r[cb]);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int cb = 0; cb < 4; ++cb)
                    if (cb * 16 < 2 * n_t) {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            acc[cb * 16 + j] += (long long)__float2int_rn(__uint_as_float(r[cb][j])) << shift;
                    }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();   // accumulators read before the next block overwrites them
        }
    }
    // epilogue: row = TMEM lane; scale by 2^{E_i + F_j - 7(S+1)} and store FP64 complex
    const int row = 32 * warp + lane;
    if (!failed && tile.m0 + row < task.M) {
        const int Ei = oa.expA[task.aexp0 + tile.m0 + row];
        const int64_t rs = task.trans ? 1 : task.ldc, cs = task.trans ? task.ldc : 1;   // row / column strides
        double* C = (double*)(g.bufs[task.c_buf] + task.c_off + (int64_t)(tile.m0 + row) * rs + (int64_t)tile.n0 * cs);
        int eB[32];   // loads ahead of the stores (see the warp-specialised kernel)
#pragma unroll
        for (int j = 0; j < 32; ++j) eB[j] = j < nval ? oa.expB[task.bexp0 + tile.n0 + j] : 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {          // accumulator columns 2j, 2j + 1: Re and Im of column j
            if (j < nval) {
                const int e = Ei + eB[j] - 7 * (S + 1);
                double2 v = make_double2(scaled_int(acc[2 * j], e), scaled_int(acc[2 * j + 1], e));
                double2* pc = reinterpret_cast<double2*>(C + 2 * (int64_t)j * cs);
                if (task.beta) { const double2 o = *pc; v.x += o.x; v.y += o.y; }
                *pc = v;
            }
        }
    }
    if (failed && tid == 0) atomicOr(oa.status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(NCOLS));
}

// ---- warp-specialised persistent variant (S <= 4) -------------------------------------------------
// One CTA per SM walks the tile list (sorted longest first) in one of two schedules, chosen per stage
// by timing when the plan is built (both give bit-identical results: the accumulation is exact):
// static (tile blockIdx.x + i gridDim.x) or a device work queue (the producer thread claims the next
// index with an atomic, one tile ahead, and passes it to the MMA thread and the epilogue warps through
// a small ring in shared memory).  Warp 0 issues the TMA loads into NST shared-memory stages, one thread of warp 1 issues the MMAs (M = 64: the M = 64 data
// path puts row i in TMEM lane 32 (i / 16) + i % 16), warps 2..17 drain the TMEM accumulators, four
// warps per lane quarter each taking 16 of the 64 accumulator columns.  Accumulation blocks (<= 8 chunks of one tile) alternate between two TMEM
// buffers, so the epilogue of one block overlaps the MMAs of the next.  Hand-offs:
//   full[st]  (TMA -> MMA, transaction bytes)     empty[st] (MMA completion -> TMA)
//   tfull[b]  (MMA completion -> epilogue)         tempty[b] (epilogue warps -> MMA)
// Tile M is a template parameter (64 or 128), chosen per stage by the autotuner: M = 64 wastes less on
// the small sector blocks, M = 128 halves the tiles (and the B reads) of blocks with more than 64 rows.
// With M = 128 every TMEM lane of a quarter holds a row (row i in lane i); three stages of
// S x (8 + 8) KB (M = 64) or two of S x (16 + 8) KB (M = 128) fit the shared memory.
template <int TMW> __host__ __device__ constexpr int ws_aboxw() { return TMW * KCH * 2; }   // bytes of one A slice box
template <int TMW> __host__ __device__ constexpr int ws_nst() { return TMW == 128 ? 2 : 3; }  // shared-memory stages
constexpr int EPIW = 16;                   // epilogue warps: four per TMEM lane quarter, 16 accumulator columns each
constexpr int THINW = 2;                   // FP64 warps for the thin sector-pair products
constexpr int kThinMaxKsteps = 8;          // a thin block's m8n8k4 steps at most (K <= 32 over all its segments)
constexpr int WS_THREADS = 64 + 32 * EPIW + 32 * THINW;
constexpr int RT = 4;                      // tile-index ring between the producer and the consumers
constexpr long kWaitWS = 1L << 22;

__device__ __forceinline__ bool mbar_wait_ws(uint32_t bar, uint32_t parity, volatile int* failed) {
    for (long i = 0; i < kWaitWS; ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if ((i & 1023) == 1023 && *failed) return false;
    }
    *failed = 1;
    return false;
}

// ---- thin sector-pair products (K3): FP64 on the warps the tensor pipeline leaves idle ---------------
// A product whose output block has fewer than thin_dim rows or columns fills a small part of a 64-row
// tensor tile, so it would cost a whole tile (TMA boxes, S(S+1)/2 MMAs per k-step, TMEM readout) for
// little work.  Such products run instead on THINW extra warps of the persistent kernel, in FP64 with
// the FP64 tensor MMA (mma.sync m8n8k4), straight from the FP64 operands (no slicing): the FP64 pipe is
// otherwise idle during the tensor pipeline, and these operands need neither slices nor TMA boxes.
// One warp computes one 8 x 8 output block over all segments of its task; items are assigned to CTAs
// at plan build, longest first onto the least loaded CTA.
__device__ __forceinline__ void dmma_f64(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
}
__device__ __forceinline__ double neg_f64(double x) { return __longlong_as_double(__double_as_longlong(x) ^ (1ll << 63)); }

__device__ __forceinline__ void thin_block(const ThinItem& it, const Task& tk, const Seg* __restrict__ segs,
                                           const GemmArgs& g, int lane) {
    const int gid = lane >> 2, tig = lane & 3;   // fragment layout of m8n8k4: A[gid][tig], B[tig][gid]
    const int r = it.m0 + gid, cb = it.n0 + gid;
    const bool rv = r < tk.M, cv = cb < tk.N;
    double cre0 = 0.0, cre1 = 0.0, cim0 = 0.0, cim1 = 0.0;
    for (int si = tk.seg_begin; si < tk.seg_end; ++si) {
        const Seg sg = segs[si];
        const cplx* __restrict__ A = g.bufs[sg.a_buf] + sg.a_off + (int64_t)r * sg.lda;
        const cplx* __restrict__ B = g.bufs[sg.b_buf] + sg.b_off;
        const bool bn = sg.opb == OPB_N, bc = sg.opb == OPB_C;
        const cplx* __restrict__ Bc = bn ? B + cb : B + (int64_t)cb * sg.ldb;   // column cb of op(B)
        const int64_t bk = bn ? sg.ldb : 1;                                         // its step along k
        double pre0 = 0.0, pre1 = 0.0, pim0 = 0.0, pim1 = 0.0;
        const bool a_real = (sg.rflags & 1) != 0, b_real = (sg.rflags & 2) != 0;   // zero imaginary products skipped
#pragma unroll 2
        for (int k0 = 0; k0 < sg.K; k0 += 4) {
            const int k = k0 + tig;
            double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
            if (rv && k < sg.K) a = A[k];
            if (cv && k < sg.K) b = Bc[(int64_t)k * bk];
            if (bc) b.y = neg_f64(b.y);
            dmma_f64(pre0, pre1, a.x, b.x);           // Re += Re a Re b - Im a Im b
            if (!a_real && !b_real) dmma_f64(pre0, pre1, neg_f64(a.y), b.y);
            if (!b_real) dmma_f64(pim0, pim1, a.x, b.y);   // Im += Re a Im b + Im a Re b
            if (!a_real) dmma_f64(pim0, pim1, a.y, b.x);
        }
        double sr = sg.scale.x, si2 = sg.scale.y;   // segment factor on the block's partial product
        if (sg.dcoef >= 0 && g.dcoef != nullptr) {   // run-time coefficient of a connection term
            const cplx d = g.dcoef[sg.dcoef];
            const double tr = sr * d.x - si2 * d.y;
            si2 = sr * d.y + si2 * d.x;
            sr = tr;
        }
        cre0 += sr * pre0 - si2 * pim0; cim0 += sr * pim0 + si2 * pre0;
        cre1 += sr * pre1 - si2 * pim1; cim1 += sr * pim1 + si2 * pre1;
    }
    if (!rv) return;
    cplx* __restrict__ C = g.bufs[tk.c_buf] + tk.c_off;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int n = it.n0 + 2 * tig + e;
        if (n < tk.N) {
            cplx* p = tk.trans ? C + (int64_t)n * tk.ldc + r : C + (int64_t)r * tk.ldc + n;
            double2 v = e ? make_double2(cre1, cim1) : make_double2(cre0, cim0);
            if (tk.beta) { const double2 o = *p; v.x += o.x; v.y += o.y; }
            *p = v;
        }
    }
}

// i-th tile of this CTA under static scheduling: blockIdx.x + i gridDim.x over the longest-first list
__device__ __forceinline__ int static_tile(uint32_t i, int ntiles, volatile int& failed) {
    const int64_t t = (int64_t)blockIdx.x + (int64_t)i * gridDim.x;
    return (t < ntiles && !failed) ? (int)t : -1;
}

template <int S, int TMW>
__global__ void __launch_bounds__(WS_THREADS, 1) k_ozaki_gemm_ws(const __grid_constant__ CUtensorMap mapA,
                                                          const __grid_constant__ CUtensorMap mapB, OzGemmArgs oa,
                                                          GemmArgs g, int ntiles, int queue, const int* skip_flag,
                                                          int skip_step) {
    pdl_enter();
    if (skip_flag != nullptr && skip_step >= *skip_flag) return;
    static_assert(S <= 4, "two TMEM buffers of S x 64 columns must fit in 512");
    static_assert(TMW == 64 || TMW == 128, "MMA M of the persistent kernel");
    constexpr uint32_t NCOLS = 512;
    constexpr int ABOXW = ws_aboxw<TMW>(), NST = ws_nst<TMW>();
    constexpr uint32_t STAGE = S * (ABOXW + BBOX);
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[NST], empty[NST], tfull[2], tempty[2], rfull[RT], rempty[RT];
    __shared__ volatile int ring[RT];
    __shared__ int sExp[EPIW][16];   // column exponents of the epilogue warps' current tile
    __shared__ uint32_t tmem_base;
    __shared__ volatile int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        failed = 0;
        for (int i = 0; i < NST; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[i])));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&tfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&tempty[i])), "r"(EPIW));
        }
        for (int i = 0; i < RT; ++i) {   // ring slot: written by the producer, read by the MMA thread and EPIW warps
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&rfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&rempty[i])), "r"(1 + EPIW));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tmem_base)), "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {   // ---------------------------------------------------------------- TMA producer
            uint32_t c = 0;
            int next = queue ? (int)atomicAdd(oa.sched, 1u) : 0;   // claimed one tile ahead
            for (uint32_t i = 0;; ++i) {
                int t;
                if (queue) {
                    const int slot = i % RT;
                    if (!mbar_wait_ws(smem_u32(&rempty[slot]), ((i / RT) & 1) ^ 1, &failed)) break;
                    t = (next < ntiles && !failed) ? next : -1;
                    ring[slot] = t;
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&rfull[slot])) : "memory");
                    if (t >= 0) next = (int)atomicAdd(oa.sched, 1u);
                } else {
                    t = static_tile(i, ntiles, failed);
                }
                if (t < 0) break;
                const OzTile tile = oa.tiles[t];
                const OzTask task = oa.tasks[tile.task];
                const int ya = task.arow0 + tile.m0, yb = task.brow0 + 2 * tile.n0;
                for (int k = 0; k < task.kchunks; ++k, ++c) {
                    const int st = c % NST;
                    if (!mbar_wait_ws(smem_u32(&empty[st]), ((c / NST) & 1) ^ 1, &failed)) break;
                    unsigned char* sA = smem + st * STAGE;
                    unsigned char* sB = sA + S * ABOXW;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(&full[st])), "r"(STAGE) : "memory");
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        tma_load(smem_u32(sA + s * ABOXW), &mapA, k * KCH, s * oa.rowsA + ya, smem_u32(&full[st]));
                        tma_load(smem_u32(sB + s * BBOX), &mapB, k * KCH, s * oa.rowsB + yb, smem_u32(&full[st]));
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ---------------------------------------------------------------- MMA issuer
            uint32_t c = 0, b = 0;
            for (uint32_t i = 0;; ++i) {
                int t;
                if (queue) {
                    const int slot = i % RT;
                    if (!mbar_wait_ws(smem_u32(&rfull[slot]), (i / RT) & 1, &failed)) break;
                    t = ring[slot];
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&rempty[slot])) : "memory");
                } else {
                    t = static_tile(i, ntiles, failed);
                }
                if (t < 0) break;
                const OzTile tile = oa.tiles[t];
                const OzTask task = oa.tasks[tile.task];
                uint32_t idesc_s[S];   // N = (S + 1 - s) 64 for A slice s (64-row B boxes; rows past 2 n_t unused)
#pragma unroll
                for (int s = 1; s <= S; ++s)
                    idesc_s[s - 1] = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(((S + 1 - s) * 64) >> 3) << 17) |
                                     ((uint32_t)(TMW >> 4) << 24);
                for (int k0 = 0; k0 < task.kchunks && !failed; k0 += kReadoutChunks, ++b) {
                    const int buf = b & 1;
                    if (!mbar_wait_ws(smem_u32(&tempty[buf]), ((b >> 1) & 1) ^ 1, &failed)) break;
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const int k1 = min(task.kchunks, k0 + kReadoutChunks);
                    for (int k = k0; k < k1; ++k, ++c) {
                        const int st = c % NST;
                        if (!mbar_wait_ws(smem_u32(&full[st]), (c / NST) & 1, &failed)) break;
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        // descriptors of the stage's first A and B boxes; every other operand is a constant
                        // offset (16-byte units) in the 14-bit start-address field, which does not overflow
                        const uint64_t da0 = desc_sw128(smem_u32(smem + st * STAGE));
                        const uint64_t db0 = desc_sw128(smem_u32(smem + st * STAGE + S * ABOXW));
                        const uint32_t tacc = tmem + (uint32_t)(buf * S * 64);
                        const bool first = k == k0;
                        // A slice s times the adjacent B slices t = 1 .. S + 1 - s in one MMA of
                        // N = (S + 1 - s) 64: box t lands in columns (s - 1 + t - 1) 64 .., the region of
                        // group g = s + t; the s = 1 MMA spans every group, so it alone starts a block
#pragma unroll
                        for (int ks = 0; ks < KCH / 16; ++ks) {
#pragma unroll
                            for (int s = 1; s <= S; ++s) {
                                const uint64_t da = da0 + (uint64_t)(((s - 1) * ABOXW + ks * 32) >> 4);
                                const uint64_t db = db0 + (uint64_t)((ks * 32) >> 4);
                                const uint32_t accum = (first && ks == 0 && s == 1) ? 0u : 1u;
                                umma(tacc + (uint32_t)((s - 1) * 64), da, db, idesc_s[s - 1], accum);
                            }
                        }
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                     :: "r"(smem_u32(&empty[st])) : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(smem_u32(&tfull[buf])) : "memory");
                }
            }
        }
    } else if (warp >= 2 + EPIW) {   // ----------------------------------------------------------- thin FP64 warps
        if (oa.tcta != nullptr) {
            const int i1 = oa.tcta[blockIdx.x + 1];
            for (int i = oa.tcta[blockIdx.x] + (warp - 2 - EPIW); i < i1; i += THINW) {
                const ThinItem it = oa.titems[i];
                thin_block(it, oa.ttasks[it.task], oa.tsegs, g, lane);
            }
        }
    } else {   // ------------------------------------------------------------------------ epilogue warps 2..17
        const int quad = warp & 3;            // TMEM lanes 32 * quad .. 32 * quad + 31 (M = 64: 16 of them hold rows)
        const int part = (warp - 2) >> 2;     // accumulator columns 16 * part .. 16 * part + 15
        const int row = (TMW == 128 ? 32 : 16) * quad + lane;
        const bool row_lane = TMW == 128 || lane < 16;   // this lane holds a row of the tile
        uint32_t b = 0;
        for (uint32_t i = 0;; ++i) {
            int t;
            if (queue) {
                const int slot = i % RT;
                if (!__all_sync(0xffffffffu, mbar_wait_ws(smem_u32(&rfull[slot]), (i / RT) & 1, &failed))) break;
                t = ring[slot];
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&rempty[slot])) : "memory");
            } else {
                t = __shfl_sync(0xffffffffu, static_tile(i, ntiles, failed), 0);
            }
            if (t < 0) break;
            const OzTile tile = oa.tiles[t];
            const OzTask task = oa.tasks[tile.task];
            const int nrem = task.N - tile.n0;
            const int nval = nrem < TNC ? nrem : TNC;
            const int n_t = (nval + 7) & ~7;
            long long acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0;
            bool ok = true;
            for (int k0 = 0; k0 < task.kchunks; k0 += kReadoutChunks, ++b) {
                const int buf = b & 1;
                // warp-uniform outcome: the warp synchronises below
                if (!__all_sync(0xffffffffu, mbar_wait_ws(smem_u32(&tfull[buf]), (b >> 1) & 1, &failed))) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                for (int gg = 2; gg <= S + 1; ++gg) {
                    const int shift = 7 * (S + 1 - gg);
                    uint32_t r[16];
                    if (part * 16 < 2 * n_t)
                        tmem_ld16(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(buf * S * 64 + (gg - 2) * 64 + part * 16), r);
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                    if (part * 16 < 2 * n_t) {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            acc[j] += (long long)__float2int_rn(__uint_as_float(r[j])) << shift;
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&tempty[buf])) : "memory");
            }
            if (!ok) break;
            // loads ahead of the stores (a load behind a store to C may not be reordered above it, so
            // loads inside the store loop would cost one memory latency each): the column exponents
            // through a per-warp row of shared memory, the beta operands eight at a time
            {   // accumulator columns 2j, 2j + 1 hold Re and Im of output column j: this warp's 16 columns
                // are output columns 8 part .. 8 part + 7
                const int j = 8 * part + (lane >> 1);
                if (lane < 16) sExp[warp - 2][lane] = j < nval ? oa.expB[task.bexp0 + tile.n0 + j] : 0;
            }
            __syncwarp();
            if (row_lane && tile.m0 + row < task.M) {
                const int Ei = oa.expA[task.aexp0 + tile.m0 + row] - 7 * (S + 1);
                const int64_t rs = task.trans ? 1 : task.ldc, cs = task.trans ? task.ldc : 1;   // row / column strides
                double* C = (double*)(g.bufs[task.c_buf] + task.c_off + (int64_t)(tile.m0 + row) * rs + (int64_t)tile.n0 * cs);
#pragma unroll
                for (int c4 = 0; c4 < 8; c4 += 4) {   // the beta operands four at a time, ahead of their stores
                    double2 old[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = 8 * part + c4 + u;
                        old[u] = (task.beta && j < nval) ? *reinterpret_cast<const double2*>(C + 2 * (int64_t)j * cs)
                                                         : make_double2(0.0, 0.0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = 8 * part + c4 + u;
                        if (j < nval) {
                            const int e = Ei + sExp[warp - 2][2 * (c4 + u)];
                            *reinterpret_cast<double2*>(C + 2 * (int64_t)j * cs) =
                                make_double2(scaled_int(acc[2 * (c4 + u)], e) + old[u].x,
                                             scaled_int(acc[2 * (c4 + u) + 1], e) + old[u].y);
                        }
                    }
                }
            }
            __syncwarp();   // sExp is rewritten for the next tile
        }
    }
    __syncwarp();   // the producer and MMA threads rejoin their warps: the barrier below waits for every thread
    __syncthreads();
    if (failed && tid == 0) atomicOr(oa.status, 1);
    if (queue && tid == 0 && atomicAdd(oa.sched + 1, 1u) == gridDim.x - 1) {   // every CTA has stopped claiming tiles
        oa.sched[0] = 0;
        oa.sched[1] = 0;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(NCOLS));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_map(tdmrg_ctx* c, CUtensorMap* m, void* base, int64_t rows, int kpad, int box_rows) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            !p) {
            cudaGetLastError();
            return fail(c, TDMRG_ECUDA, "cuTensorMapEncodeTiled unavailable");
        }
        fn = (EncodeTiledFn)p;
    }
    cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
    cuuint32_t box[2] = {(cuuint32_t)KCH, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, TDMRG_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return TDMRG_OK;
}

template <int S>
cudaError_t gemm_attr() {
    if constexpr (S <= 4) {
        const size_t s64 = (size_t)ws_nst<64>() * S * (ws_aboxw<64>() + BBOX) + 1024;
        const size_t s128 = (size_t)ws_nst<128>() * S * (ws_aboxw<128>() + BBOX) + 1024;
        cudaError_t e = cudaFuncSetAttribute(k_ozaki_gemm_ws<S, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_ozaki_gemm_ws<S, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s128);
        return e;
    } else {
        const size_t smem = (size_t)S * (ABOX + BBOX) + 1024;
        return cudaFuncSetAttribute(k_ozaki_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
}

int g_num_sms = 0;

template <int S>
cudaError_t gemm_launch(const OzStage& st, const GemmArgs& g, cudaStream_t s, const int* skip_flag, int skip_step) {
    if constexpr (S <= 4) {
        OzGemmArgs a = st.args;
        if (st.tmw == 128) {
            const size_t smem = (size_t)ws_nst<128>() * S * (ws_aboxw<128>() + BBOX) + 1024;
            a.tiles = st.d_tiles128;
            launch_pdl(k_ozaki_gemm_ws<S, 128>, std::max(1, st.grid), WS_THREADS, smem, s, st.mapA128, st.mapB, a, g,
                       (int)st.tiles128.size(), st.queue, skip_flag, skip_step);
        } else {
            const size_t smem = (size_t)ws_nst<64>() * S * (ws_aboxw<64>() + BBOX) + 1024;
            launch_pdl(k_ozaki_gemm_ws<S, 64>, std::max(1, st.grid), WS_THREADS, smem, s, st.mapA, st.mapB, a, g,
                       (int)st.tiles.size(), st.queue, skip_flag, skip_step);
        }
        return cudaGetLastError();
    }
    const size_t smem = (size_t)S * (ABOX + BBOX) + 1024;
    launch_pdl(k_ozaki_gemm<S>, (int)st.tiles.size(), 128, smem, s, st.mapA, st.mapB, st.args, g, skip_flag, skip_step);
    return cudaGetLastError();
}

cudaError_t slice_launch(const OzSliceArgs& sa, const GemmArgs& g, cudaStream_t s, const int* skip_flag, int skip_step) {
    if (sa.nvec_total <= 0) return cudaSuccess;
    const int grid = sa.nvec_total;   // one CTA per vector
    switch (sa.S) {
        case 2: launch_pdl(k_slice<2>, grid, kSliceCT, 0, s, sa, g, skip_flag, skip_step); break;
        case 3: launch_pdl(k_slice<3>, grid, kSliceCT, 0, s, sa, g, skip_flag, skip_step); break;
        case 4: launch_pdl(k_slice<4>, grid, kSliceCT, 0, s, sa, g, skip_flag, skip_step); break;
        case 5: launch_pdl(k_slice<5>, grid, kSliceCT, 0, s, sa, g, skip_flag, skip_step); break;
        case 6: launch_pdl(k_slice<6>, grid, kSliceCT, 0, s, sa, g, skip_flag, skip_step); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
int upload_vec(tdmrg_ctx* c, const std::vector<T>& v, T** d, const char* what) {
    *d = nullptr;
    if (v.empty()) return TDMRG_OK;
    int rc = dev_alloc(c, (void**)d, v.size() * sizeof(T), what);
    if (rc) return rc;
    return cuda_check(c, cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), what);
}

}  // namespace

void release_oz(tdmrg_ctx* c, OzPlan& oz) {
    for (OzStage& st : oz.st) {
        dev_free(c, st.d_tasks, st.tasks.size() * sizeof(OzTask));
        dev_free(c, st.d_tiles, st.tiles.size() * sizeof(OzTile));
        dev_free(c, st.d_tiles128, st.tiles128.size() * sizeof(OzTile));
        dev_free(c, st.d_ajobs, st.ajobs.size() * sizeof(OzSliceJob));
        dev_free(c, st.d_bjobs, st.bjobs.size() * sizeof(OzSliceJob));
        dev_free(c, st.d_avjob, st.avjob.size() * sizeof(int));
        dev_free(c, st.d_bvjob, st.bvjob.size() * sizeof(int));
        dev_free(c, st.d_asegs, st.asegs.size() * sizeof(Seg));
        dev_free(c, st.d_bsegs, st.bsegs.size() * sizeof(Seg));
        dev_free(c, st.panelA, st.panel_bytes_a);
        dev_free(c, st.panelB, st.panel_bytes_b);
        dev_free(c, st.expA, st.exp_bytes_a);
        dev_free(c, st.expB, st.exp_bytes_b);
        dev_free(c, st.d_sched, 2 * sizeof(unsigned));
        dev_free(c, st.d_ttasks, st.ttasks.size() * sizeof(Task));
        dev_free(c, st.d_tsegs, st.tsegs.size() * sizeof(Seg));
        dev_free(c, st.d_titems, st.titems.size() * sizeof(ThinItem));
        dev_free(c, st.d_tcta, st.tcta.size() * sizeof(int));
        st = OzStage();
    }
    oz.status = nullptr;   // owned by the context
    oz.ready = false;
}

// Tile schedule of each stage by timing (the autotuner of the grouped launch): the persistent kernel
// runs once per candidate on temporary input and output buffers (its time does not depend on the
// values), and the static schedule is kept unless the work queue is at least 3% faster.  Every
// schedule computes the same exact integer sums, so the choice never changes a result.
static int autotune_oz(tdmrg_ctx* c, Plan* p) {
    OzPlan& oz = p->oz;
    if (oz.S > 4) return TDMRG_OK;   // only the persistent kernel has schedules and tile shapes
    const bool fix_q = c->schedule >= 0, fix_m = c->tile_m > 0;   // fixed by tdmrg_set_schedule / tdmrg_set_tile_m
    for (OzStage& st : oz.st) {
        st.queue = fix_q ? c->schedule : 0;
        st.tmw = (fix_m && c->tile_m == 128 && !st.tiles128.empty()) ? 128 : 64;
    }
    if (fix_q && fix_m) return TDMRG_OK;
    cplx *tin = nullptr, *tout = nullptr;
    const size_t bin = (size_t)std::max<int64_t>(p->n_in, 1) * sizeof(cplx), bout = (size_t)std::max<int64_t>(p->n_out, 1) * sizeof(cplx);
    int rc = dev_alloc(c, (void**)&tin, bin, "autotuning buffers");
    if (!rc) rc = dev_alloc(c, (void**)&tout, bout, "autotuning buffers");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc) rc = cuda_check(c, cudaEventCreate(&e0), "autotuning events");
    if (!rc) rc = cuda_check(c, cudaEventCreate(&e1), "autotuning events");
    GemmArgs g{};
    g.bufs[BUF_OPS] = c->pool;
    g.bufs[BUF_IN] = tin;
    g.bufs[BUF_SCRATCH] = c->scratch;
    g.bufs[BUF_OUT] = tout;
    g.dscale = c->dscale;
    auto launch = [&](const OzStage& st) {
        switch (oz.S) {
            case 2: return gemm_launch<2>(st, g, c->stream, nullptr, 0);
            case 3: return gemm_launch<3>(st, g, c->stream, nullptr, 0);
            default: return gemm_launch<4>(st, g, c->stream, nullptr, 0);
        }
    };
    // per stage: every allowed (tile M, schedule) timed; the default (M = 64, static) is kept unless
    // another is at least 3 % faster.  Every choice computes the same exact integer sums.
    for (int stg = 0; stg < 2 && !rc; ++stg) {
        OzStage& st = oz.st[stg];
        if (st.tasks.empty()) continue;
        std::vector<std::pair<int, int>> cand;
        for (int m : {64, 128}) {
            if (m == 128 && st.tiles128.empty()) continue;
            if (fix_m && m != st.tmw) continue;
            for (int q : {0, 1}) {
                if (fix_q && q != c->schedule) continue;
                cand.push_back({m, q});
            }
        }
        float best = 0.f;
        std::pair<int, int> pick = cand.front();
        for (size_t k = 0; k < cand.size() && !rc; ++k) {
            st.tmw = cand[k].first;
            st.queue = cand[k].second;
            float ms = 0.f;
            cudaError_t e = launch(st);   // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch(st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            rc = cuda_check(c, e, "autotuning");
            if (k == 0 || ms < 0.97f * best) { best = ms; pick = cand[k]; }
        }
        st.tmw = pick.first;
        st.queue = pick.second;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(c, tin, bin);
    dev_free(c, tout, bout);
    return rc;
}

// Build the tensor-core form of the two stages of a plan.  Tasks that the tensor path does not take
// (no segments, several stage-1 segments, K above the exact-accumulation limits) stay in p.thin[st]
// and run on the FP64 kernel.
int build_oz(tdmrg_ctx* c, Plan* p, int S) {
    OzPlan& oz = p->oz;
    release_oz(c, oz);
    oz.S = S;
    oz.status = c->dstatus;
    const int tm = S <= 4 ? 64 : TM;   // MMA M of the kernel that runs this precision (S <= 4: also an M = 128 list)
    int rc = TDMRG_OK;
    for (int stg = 0; stg < 2; ++stg) {
        const TaskList& tl = stg == 0 ? p->stage1 : p->stage2;
        TaskList& thin = p->thin[stg];
        release(c, thin);
        thin.tasks.clear(); thin.segs.clear();
        OzStage& st = oz.st[stg];
        std::map<int64_t, int> pair_row;   // stage 1: Psi block offset -> A panel row
        int rowsA = 0, rowsB = 0, kmax = 0;
        for (size_t t = 0; t < tl.tasks.size(); ++t) {
            const Task& tk = tl.tasks[t];
            const int nseg = tk.seg_end - tk.seg_begin;
            int ktot = 0;
            bool dev_scale = false;
            for (int s = tk.seg_begin; s < tk.seg_end; ++s) { ktot += tl.segs[s].K; dev_scale |= tl.segs[s].dscale >= 0; }
            // thin product: on the FP64 warps of the persistent kernel (S <= 4), in 8 x 8 output blocks, if one
            // block's FP64 chain is short (GB300 runs an m8n8k4 FP64 MMA in ~640 cycles of a sub-partition)
            int ksteps_all = 0;
            for (int s = tk.seg_begin; s < tk.seg_end; ++s) ksteps_all += (tl.segs[s].K + 3) / 4;
            if (S <= 4 && c->thin_dim > 0 && nseg > 0 && !dev_scale && std::min(tk.M, tk.N) < c->thin_dim &&
                ksteps_all <= kThinMaxKsteps) {
                Task nt = tk;
                nt.seg_begin = (int)st.tsegs.size();
                for (int s = tk.seg_begin; s < tk.seg_end; ++s) st.tsegs.push_back(tl.segs[s]);
                nt.seg_end = (int)st.tsegs.size();
                const int ti = (int)st.ttasks.size();
                st.ttasks.push_back(nt);
                int ksteps = 0;   // m8n8k4 steps of one block over all segments
                for (int s = tk.seg_begin; s < tk.seg_end; ++s) ksteps += (tl.segs[s].K + 3) / 4;
                for (int m0 = 0; m0 < tk.M; m0 += 8)
                    for (int n0 = 0; n0 < tk.N; n0 += 8) st.titems.push_back({ti, m0, n0, std::max(ksteps, 1)});
                st.thin_flops += 8.0 * tk.M * tk.N * (double)ktot;
                continue;
            }
            // a stage-1 segment with a run-time coefficient would need its static operator slices redone at
            // every product: such tasks stay on the FP64 kernel
            bool run_time = false;
            for (int s = tk.seg_begin; s < tk.seg_end; ++s) run_time |= tl.segs[s].dcoef >= 0;
            const bool ok = nseg > 0 && (stg == 1 || nseg == 1) && 2 * ktot <= 4096 && !(stg == 0 && run_time);
            if (!ok) {   // FP64 kernel
                Task nt = tk;
                nt.seg_begin = (int)thin.segs.size();
                for (int s = tk.seg_begin; s < tk.seg_end; ++s) thin.segs.push_back(tl.segs[s]);
                nt.seg_end = (int)thin.segs.size();
                thin.tasks.push_back(nt);
                continue;
            }
            OzTask ot{};
            ot.c_off = tk.c_off; ot.c_buf = tk.c_buf; ot.ldc = tk.ldc; ot.M = tk.M; ot.N = tk.N; ot.beta = tk.beta;
            ot.trans = tk.trans;
            // every A segment real (stage 2, real operators with real factors): A' = [Re A | 0], and the first
            // halves of the B' rows hold Re b and Im b, so only the first ktot of the real K are used
            bool all_a_real = stg == 1;
            for (int s = tk.seg_begin; s < tk.seg_end; ++s) all_a_real &= (tl.segs[s].rflags & 1) != 0;
            ot.kchunks = ((all_a_real ? ktot : 2 * ktot) + KCH - 1) / KCH;
            kmax = std::max(kmax, 2 * ktot);
            // A operand
            if (stg == 0) {   // A = Psi_{q'}: one dynamic row-sliced panel per input pair, shared by its tasks
                const Seg& sg = tl.segs[tk.seg_begin];
                auto it = pair_row.find(sg.a_off);
                if (it == pair_row.end()) {
                    Seg js = sg;
                    js.scale = make_double2(1.0, 0.0);
                    OzSliceJob j{};
                    j.role = 0; j.nvec = tk.M; j.seg_begin = (int)st.asegs.size(); j.seg_end = j.seg_begin + 1;
                    j.row0 = rowsA; j.exp0 = rowsA; j.ktot = sg.K; j.use_scale = 0;
                    st.asegs.push_back(js);
                    st.ajobs.push_back(j);
                    it = pair_row.emplace(sg.a_off, rowsA).first;
                    rowsA += tk.M;
                }
                ot.arow0 = it->second; ot.aexp0 = it->second;
            } else {          // A = [ops of all segments]: static, sliced once, with the segment factors
                              // folded in, unless the coefficients are read at run time (then on B)
                OzSliceJob j{};
                j.role = 0; j.nvec = tk.M; j.seg_begin = (int)st.asegs.size();
                for (int s = tk.seg_begin; s < tk.seg_end; ++s) st.asegs.push_back(tl.segs[s]);
                j.seg_end = (int)st.asegs.size();
                j.row0 = rowsA; j.exp0 = rowsA; j.ktot = ktot; j.use_scale = c->dcoef == nullptr ? 1 : 0;
                st.ajobs.push_back(j);
                ot.arow0 = rowsA; ot.aexp0 = rowsA;
                rowsA += tk.M;
            }
            // B operand: columns of op(B), K-concatenated over segments
            {
                OzSliceJob j{};
                j.role = 1; j.nvec = tk.N; j.seg_begin = (int)st.bsegs.size();
                for (int s = tk.seg_begin; s < tk.seg_end; ++s) st.bsegs.push_back(tl.segs[s]);
                j.seg_end = (int)st.bsegs.size();
                j.row0 = rowsB; j.exp0 = st.ncolsB; j.ktot = ktot;
                // the segment factor (coefficient and fermion sign) goes on the static operator: B of stage 1,
                // A of stage 2; with run-time coefficients the stage-2 factors go on B, the intermediates
                // sliced at every product, so that they may change between products
                j.use_scale = (stg == 0 || c->dcoef != nullptr) ? 1 : 0;
                st.bjobs.push_back(j);
                ot.brow0 = rowsB; ot.bexp0 = st.ncolsB;
                const int full = tk.N / TNC, rem = tk.N % TNC;
                rowsB += 2 * TNC * full + 2 * ((rem + 7) & ~7);
                st.ncolsB += tk.N;
            }
            const int ti = (int)st.tasks.size();
            st.tasks.push_back(ot);
            for (int m0 = 0; m0 < tk.M; m0 += tm)
                for (int n0 = 0; n0 < tk.N; n0 += TNC) st.tiles.push_back({ti, m0, n0, (int)(std::min(tm, tk.M - m0) * std::min(TNC, tk.N - n0)) * ot.kchunks});
            if (S <= 4)
                for (int m0 = 0; m0 < tk.M; m0 += 128)
                    for (int n0 = 0; n0 < tk.N; n0 += TNC)
                        st.tiles128.push_back({ti, m0, n0, (int)(std::min(128, tk.M - m0) * std::min(TNC, tk.N - n0)) * ot.kchunks});
        }
        std::stable_sort(st.tiles.begin(), st.tiles.end(), [](const OzTile& a, const OzTile& b) { return a.cost > b.cost; });
        std::stable_sort(st.tiles128.begin(), st.tiles128.end(), [](const OzTile& a, const OzTile& b) { return a.cost > b.cost; });
        // persistent grid: one CTA per SM when thin items exist (their warps ride along), else one per tile
        st.grid = st.titems.empty() ? std::max(1, std::min((int)st.tiles.size(), c->num_sms)) : c->num_sms;
        if (!st.titems.empty()) {   // thin items: longest first onto the least loaded CTA, grouped by CTA
            std::stable_sort(st.titems.begin(), st.titems.end(),
                             [](const ThinItem& a, const ThinItem& b) { return a.cost > b.cost; });
            std::vector<int64_t> load(st.grid, 0);
            std::vector<std::vector<ThinItem>> per(st.grid);
            for (const ThinItem& it : st.titems) {
                const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                load[b] += it.cost;
                per[b].push_back(it);
            }
            st.titems.clear();
            st.tcta.assign(1, 0);
            for (const auto& v : per) {
                st.titems.insert(st.titems.end(), v.begin(), v.end());
                st.tcta.push_back((int)st.titems.size());
            }
        }
        // panels: rows padded so that every TMA box (tm rows for A, 64 for B) stays inside the plane
        st.rowsA = rowsA + (S <= 4 ? 128 : tm);
        st.rowsB = rowsB + 2 * TNC;
        st.kpad = std::max(KCH, (kmax + KCH - 1) / KCH * KCH);
        st.panel_bytes_a = (size_t)S * st.rowsA * st.kpad * 2;
        st.panel_bytes_b = (size_t)S * st.rowsB * st.kpad * 2;
        st.exp_bytes_a = (size_t)std::max(rowsA, 1) * sizeof(int);
        st.exp_bytes_b = (size_t)std::max(st.ncolsB, 1) * sizeof(int);
        st.avjob.clear(); st.bvjob.clear();
        for (size_t j = 0, pre = 0; j < st.ajobs.size(); ++j) {
            st.ajobs[j].vec_prefix = (int)pre; pre += st.ajobs[j].nvec;
            st.avjob.insert(st.avjob.end(), st.ajobs[j].nvec, (int)j);
        }
        for (size_t j = 0, pre = 0; j < st.bjobs.size(); ++j) {
            st.bjobs[j].vec_prefix = (int)pre; pre += st.bjobs[j].nvec;
            st.bvjob.insert(st.bvjob.end(), st.bjobs[j].nvec, (int)j);
        }
        if (!st.titems.empty()) {
            rc = upload_vec(c, st.ttasks, &st.d_ttasks, "thin tasks");
            if (!rc) rc = upload_vec(c, st.tsegs, &st.d_tsegs, "thin segments");
            if (!rc) rc = upload_vec(c, st.titems, &st.d_titems, "thin items");
            if (!rc) rc = upload_vec(c, st.tcta, &st.d_tcta, "thin items");
            if (rc) return rc;
        }
        st.args.ttasks = st.d_ttasks; st.args.tsegs = st.d_tsegs; st.args.titems = st.d_titems; st.args.tcta = st.d_tcta;
        st.args.status = oz.status;
        if (!st.tasks.empty() || !st.titems.empty()) {   // work-queue counters (also for a stage of thin items only)
            rc = dev_alloc(c, (void**)&st.d_sched, 2 * sizeof(unsigned), "ozaki work queue");
            if (!rc) rc = cuda_check(c, cudaMemset(st.d_sched, 0, 2 * sizeof(unsigned)), "ozaki work queue");
            if (rc) return rc;
            st.args.sched = st.d_sched;
        }
        if (!st.tasks.empty()) {
            rc = dev_alloc(c, (void**)&st.panelA, st.panel_bytes_a, "ozaki panels");
            if (!rc) rc = dev_alloc(c, (void**)&st.panelB, st.panel_bytes_b, "ozaki panels");
            if (!rc) rc = dev_alloc(c, (void**)&st.expA, st.exp_bytes_a, "ozaki exponents");
            if (!rc) rc = dev_alloc(c, (void**)&st.expB, st.exp_bytes_b, "ozaki exponents");
            if (!rc) rc = cuda_check(c, cudaMemset(st.panelA, 0, st.panel_bytes_a), "ozaki panels");
            if (!rc) rc = cuda_check(c, cudaMemset(st.panelB, 0, st.panel_bytes_b), "ozaki panels");
            if (!rc) rc = upload_vec(c, st.tasks, &st.d_tasks, "ozaki tasks");
            if (!rc) rc = upload_vec(c, st.tiles, &st.d_tiles, "ozaki tiles");
            if (!rc && !st.tiles128.empty()) rc = upload_vec(c, st.tiles128, &st.d_tiles128, "ozaki tiles");
            if (!rc) rc = upload_vec(c, st.ajobs, &st.d_ajobs, "ozaki slice jobs");
            if (!rc) rc = upload_vec(c, st.bjobs, &st.d_bjobs, "ozaki slice jobs");
            if (!rc && !st.avjob.empty()) rc = upload_vec(c, st.avjob, &st.d_avjob, "ozaki slice jobs");
            if (!rc && !st.bvjob.empty()) rc = upload_vec(c, st.bvjob, &st.d_bvjob, "ozaki slice jobs");
            if (!rc) rc = upload_vec(c, st.asegs, &st.d_asegs, "ozaki slice segments");
            if (!rc) rc = upload_vec(c, st.bsegs, &st.d_bsegs, "ozaki slice segments");
            if (!rc) rc = encode_map(c, &st.mapA, st.panelA, (int64_t)S * st.rowsA, st.kpad, tm);
            if (!rc && S <= 4) rc = encode_map(c, &st.mapA128, st.panelA, (int64_t)S * st.rowsA, st.kpad, 128);
            if (!rc) rc = encode_map(c, &st.mapB, st.panelB, (int64_t)S * st.rowsB, st.kpad, 2 * TNC);
            if (rc) return rc;
            st.args.tasks = st.d_tasks; st.args.tiles = st.d_tiles;
            st.args.expA = st.expA; st.args.expB = st.expB;
            st.args.rowsA = st.rowsA; st.args.rowsB = st.rowsB;
            auto mk = [&](OzSliceArgs& sa, const std::vector<OzSliceJob>& jobs, OzSliceJob* dj, const int* dv, Seg* ds,
                          __nv_bfloat16* panel, int* exps, int rows) {
                sa.jobs = dj; sa.vjob = dv; sa.njobs = (int)jobs.size(); sa.segs = ds; sa.panel = panel; sa.exps = exps;
                sa.rows = rows; sa.kpad = st.kpad; sa.S = S;
                sa.nvec_total = jobs.empty() ? 0 : jobs.back().vec_prefix + jobs.back().nvec;
            };
            mk(st.sliceA, st.ajobs, st.d_ajobs, st.d_avjob, st.d_asegs, st.panelA, st.expA, st.rowsA);
            mk(st.sliceB, st.bjobs, st.d_bjobs, st.d_bvjob, st.d_bsegs, st.panelB, st.expB, st.rowsB);
        }
        if (!thin.tasks.empty()) {
            make_tiles(thin, kTileF64, kTileF64, kSplitK);
            rc = upload(c, thin);
            if (rc) return rc;
        }
    }
    g_num_sms = c->num_sms;
    {   // shared-memory opt-in of the GEMM for this S (set here, outside any stream capture)
        cudaError_t e = S == 2 ? gemm_attr<2>() : S == 3 ? gemm_attr<3>() : S == 4 ? gemm_attr<4>()
                      : S == 5 ? gemm_attr<5>() : gemm_attr<6>();
        rc = cuda_check(c, e, "ozaki shared memory");
        if (rc) return rc;
    }
    // static operands: stage-1 B (operators, scales folded) and stage-2 A (operators, scales folded)
    GemmArgs g{};
    g.bufs[BUF_OPS] = c->pool;
    if (!oz.st[0].tasks.empty()) {
        rc = cuda_check(c, slice_launch(oz.st[0].sliceB, g, c->stream, nullptr, 0), "ozaki static slices");
        if (rc) return rc;
    }
    if (!oz.st[1].tasks.empty()) {
        rc = cuda_check(c, slice_launch(oz.st[1].sliceA, g, c->stream, nullptr, 0), "ozaki static slices");
        if (rc) return rc;
    }
    rc = cuda_check(c, cudaStreamSynchronize(c->stream), "ozaki static slices");
    if (!rc) rc = autotune_oz(c, p);
    if (rc) return rc;
    oz.ready = true;
    return TDMRG_OK;
}

int run_oz(tdmrg_ctx* c, const Plan& p, const cplx* in, cplx* out, const int* skip_flag, int skip_step) {
    const OzPlan& oz = p.oz;
    GemmArgs g{};
    g.bufs[BUF_OPS] = c->pool;
    g.bufs[BUF_IN] = const_cast<cplx*>(in);
    g.bufs[BUF_SCRATCH] = c->scratch;
    g.bufs[BUF_OUT] = out;
    g.dscale = c->dscale;
    g.dcoef = c->dcoef;
    cudaStream_t s = c->stream;
    for (int stg = 0; stg < 2; ++stg) {
        const OzStage& st = oz.st[stg];
        cudaError_t e = cudaSuccess;
        if (!st.tasks.empty() || !st.titems.empty()) {
            if (!st.tasks.empty()) {
                e = slice_launch(stg == 0 ? st.sliceA : st.sliceB, g, s, skip_flag, skip_step);
                c->launches++;
            }
            if (e == cudaSuccess) {
                switch (oz.S) {
                    case 2: e = gemm_launch<2>(st, g, s, skip_flag, skip_step); break;
                    case 3: e = gemm_launch<3>(st, g, s, skip_flag, skip_step); break;
                    case 4: e = gemm_launch<4>(st, g, s, skip_flag, skip_step); break;
                    case 5: e = gemm_launch<5>(st, g, s, skip_flag, skip_step); break;
                    case 6: e = gemm_launch<6>(st, g, s, skip_flag, skip_step); break;
                    default: e = cudaErrorInvalidValue;
                }
                c->launches++;
            }
        }
        const TaskList& thin = p.thin[stg];
        if (e == cudaSuccess && !thin.tiles.empty()) {
            GemmArgs a = g;
            a.tasks = thin.d_tasks; a.segs = thin.d_segs; a.tiles = thin.d_tiles; a.ntiles = (int)thin.tiles.size();
            a.partials = thin.d_partials; a.counters = thin.d_counters;
            e = launch_gemm_f64(a, s, skip_flag, skip_step);
            c->launches++;
        }
        int rc = cuda_check(c, e, "ozaki superblock product launch");
        if (rc) return rc;
    }
    return TDMRG_OK;
}

int oz_status(tdmrg_ctx* c, const Plan& p, int* status) {
    *status = 0;
    if (!p.oz.status) return TDMRG_OK;
    return cuda_check(c, cudaMemcpy(status, p.oz.status, sizeof(int), cudaMemcpyDeviceToHost), "ozaki status");
}

}  // namespace tdmrg
