// Krylov time evolution on the device (Sec. II.A, Eq. lanczosevolution; Sec. II.C,
// Eq. lanczosevolution2; time targets of Sec. II.B).
//
// Lanczos is started from phi itself: v_0 = phi / ||phi||.  Step j: w = H v_j (grouped superblock
// product), alpha_j = Re <v_j|w>, then two classical Gram-Schmidt passes against v_0..v_j
// (the first pass also removes the alpha_j v_j and beta_j v_{j-1} components; its dots in FP32, the second
// pass in FP64 removes what they leave, and alpha_j is the sum of both passes' coefficients),
// beta_{j+1} = ||w||, v_{j+1} = w / beta_{j+1}, all in one cooperative launch per step with two grid
// barriers; the recursion stops at n_K vectors or when beta_{j+1} <= tol * max(1, |alpha_j|).  Then the
// coefficients c_x = ||phi|| e^{-i T t_x} e_0 (= ||phi|| [S^dag e^{-i D t_x} S]_{.,0} with T = S^dag D S)
// are computed on the tridiagonal itself (Taylor series on short substeps, FP64; for equally spaced
// times by powers of the step exponential) and the targets phi(t_x) = sum_k v_k c_x[k] are formed in
// one pass over V.  The vectors, alpha and beta are FP64-accurate and stay on the device; reductions use
// a fixed grid and a fixed summation order, so results do not depend on scheduling.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace tdmrg {
namespace {

constexpr int NB = kRedBlocks;   // reduction blocks
constexpr int kCoefWords = (16 + 32) * 32;   // Krylov coefficients of 16 targets + step exponential columns
constexpr int kBarWords = 4;                  // grid barrier counter, exponential ticket
constexpr int NT = 256;          // threads per reduction block
enum { T_ALPHA = 0, T_BETA = 32, T_BETA0 = 64, T_RESID = 65, T_ERR = 66, T_EMIN = 67 };

__device__ __forceinline__ void chunk_of(int64_t n, int64_t& lo, int64_t& hi) {
    const int64_t ch = (n + NB - 1) / NB;
    lo = min(n, (int64_t)blockIdx.x * ch);
    hi = min(n, lo + ch);
}

// Deterministic block sum of a double2 (fixed butterfly, fixed warp order).
__device__ double2 block_sum(double2 v) {
    __shared__ double2 sh[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < NT / 32; ++k) { s.x += sh[k].x; s.y += sh[k].y; }
    return s;   // every thread holds the block total
}

// Sum of part[0..NB-1] by one warp in a fixed order (identical in every block that calls it).
__device__ double2 warp_total(const double2* __restrict__ part) {
    const int l = threadIdx.x & 31;
    double2 s = make_double2(0.0, 0.0);
    for (int b = l; b < NB; b += 32) { s.x += part[b].x; s.y += part[b].y; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    return s;
}

// h[k] = sum of partials of vector k, for k < nv; every block computes the same values.
__device__ void reduce_coeffs(const double2* __restrict__ part, int nv, double2* h) {
    const int w = threadIdx.x >> 5;
    for (int k = w; k < nv; k += NT / 32) {
        double2 s = warp_total(part + (int64_t)k * NB);
        if ((threadIdx.x & 31) == 0) h[k] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ double2 cdotc(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__global__ void __launch_bounds__(NT) k_norm2(const cplx* __restrict__ x, int64_t n, double2* __restrict__ part) {
    pdl_enter();
    int64_t lo, hi;
    chunk_of(n, lo, hi);
    double s = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += NT) { const double2 v = x[i]; s += v.x * v.x + v.y * v.y; }
    double2 t = block_sum(make_double2(s, 0.0));
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) k_init_v0(const cplx* __restrict__ phi, int64_t n, const double2* __restrict__ part,
                                                 cplx* __restrict__ v0, double* __restrict__ tri, int* __restrict__ flags,
                                                 int nk) {
    pdl_enter();
    __shared__ double2 h[1];
    reduce_coeffs(part, 1, h);
    const double b0 = sqrt(h[0].x);
    const double inv = b0 > 0.0 ? 1.0 / b0 : 0.0;
    int64_t lo, hi;
    chunk_of(n, lo, hi);
    for (int64_t i = lo + threadIdx.x; i < hi; i += NT) { const double2 v = phi[i]; v0[i] = make_double2(v.x * inv, v.y * inv); }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        tri[T_BETA0] = b0;
        tri[T_RESID] = 0.0;
        flags[0] = b0 > 0.0 ? nk : 0;
    }
}

// ---- one Lanczos orthogonalisation step in a single cooperative launch -----------------------
// Two grid barriers separate: (A) the first-pass dots h1_k = <v_k|w>; (B) w' = w - sum h1_k v_k, the
// second-pass dots h2_k = <v_k|w'> and ||w'||^2; (C) beta = ||w' - sum h2_k v_k|| and
// v_{j+1} = (w' - sum h2_k v_k) / beta.  Since h2 holds the projections of w' on orthonormal v_k,
// ||w' - sum h2_k v_k||^2 = ||w'||^2 - sum |h2_k|^2 (h2 is at rounding level after the first pass, so
// the difference loses nothing), which saves the barrier of a separate norm pass.  Every block
// reduces the partials of all blocks in the same fixed order, so results do not depend on
// scheduling.  FP64 throughput per SM is low on this GPU, so the warp reductions are
// reduce-scatter (16 FP64 adds for 16 values instead of 80).  The barrier spins are bounded: when one
// runs out the kernel sets a status bit and finishes.
constexpr int OB = 256;   // threads per block of the fused kernel
constexpr long kBarrierSpin = 1L << 24;

// Segmented mode: the vector holds independent problems side by side (a direct sum of superblocks);
// CTA b works on elements [lo_b, hi_b) of segment seg_b, and each segment has its own partial sums,
// tridiagonal (kTriStride doubles), flags (kFlagStride ints) and coefficients (kCoefStride).
constexpr int kTriStride = 128, kFlagStride = 4, kCoefStride = 16 * 32;
struct SegTab {
    const int* cta_seg;
    const int64_t* cta_lo;
    const int64_t* cta_hi;
    const int* seg_cta0;   // first CTA of each segment; seg_cta0[nseg] = the grid
    int nseg;
};

struct OrthArgs {
    const cplx* V;
    cplx* w;
    int64_t n;
    int nv, j, nk;
    double tol;
    double2* partA;
    double2* partB;
    double* tri;
    int* flags;
    unsigned* bar;     // [0] grid barrier counter (top bit flips at each barrier)
    int* status;
    SegTab seg;        // seg.nseg == 0: one problem over the whole vector
};

// Grid barrier of the co-resident (cooperative) grid on one counter word whose low 31 bits stay zero:
// block 0 adds 2^31 - (G - 1), every other block 1, so the top bit flips exactly when the last block
// arrives, and each block waits until the top bit differs from the value it saw at its own arrival.  The
// last arrival releases everyone directly (no reset, no second word).  Bounded wait: status bit 2.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void grid_barrier(unsigned* bar, int* status) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
        __threadfence();
        const unsigned old = atomicAdd(bar, add);
        long it = 0;
        while (((old ^ ld_acquire_u32(bar)) & 0x80000000u) == 0u) {
            if (++it > kBarrierSpin) { atomicOr(status, 2); break; }
        }
        __threadfence();
    }
    __syncthreads();
}

// Block sums of NK complex values in a fixed order; the result is in out[0..NK-1].  Warp level:
// reduce-scatter over ND = 2 * pow2ceil(NK) doubles (log2 ND halving levels, then a butterfly over the
// remaining lane bits), after which lane l holds the warp total of double l >> (5 - log2 ND).
template <int NK>
__device__ void block_sum(double2 (&v)[NK], double* sh /* [OB/32][16] */, double2* out) {
    constexpr int ND = NK <= 1 ? 2 : NK <= 2 ? 4 : NK <= 4 ? 8 : 16;
    constexpr int LV = ND == 2 ? 1 : ND == 4 ? 2 : ND == 8 ? 3 : 4;
    double d[ND];
#pragma unroll
    for (int k = 0; k < ND / 2; ++k) {
        d[2 * k] = k < NK ? v[k < NK ? k : 0].x : 0.0;
        d[2 * k + 1] = k < NK ? v[k < NK ? k : 0].y : 0.0;
    }
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int lv = 0; lv < LV; ++lv) {
        const int half = ND >> (lv + 1), o = 16 >> lv;
        const bool up = (l & o) != 0;   // keep the upper half of the remaining values
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const double lo_v = d[i], hi_v = d[i + half];
            const double send = up ? lo_v : hi_v;
            d[i] = (up ? hi_v : lo_v) + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = 16 >> LV; o > 0; o >>= 1) d[0] += __shfl_xor_sync(0xffffffffu, d[0], o);
    __syncthreads();
    if ((l & ((32 >> LV) - 1)) == 0) sh[w * 16 + (l >> (5 - LV))] = d[0];
    __syncthreads();
    if (threadIdx.x < 2 * NK) {
        double s = 0.0;
        for (int ww = 0; ww < OB / 32; ++ww) s += sh[ww * 16 + threadIdx.x];
        reinterpret_cast<double*>(out)[threadIdx.x] = s;
    }
    __syncthreads();
}

// Deterministic block sum of one double (result in every thread).
__device__ double block_sum1(double x, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < OB / 32; ++k) s += sh[k];
    __syncthreads();
    return s;
}

// partials[k * gridDim + b] for k < nv and b in [b0, b1)  ->  every block's h[k] (same order everywhere)
__device__ void sum_partials(const double2* __restrict__ part, int nv, double2* h, int b0 = 0, int b1 = -1) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (b1 < 0) b1 = (int)gridDim.x;
    for (int k = w; k < nv; k += OB / 32) {
        double2 s = make_double2(0.0, 0.0);
        for (int b = b0 + l; b < b1; b += 32) { s.x += part[(int64_t)k * gridDim.x + b].x; s.y += part[(int64_t)k * gridDim.x + b].y; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
        if (l == 0) h[k] = s;
    }
    __syncthreads();
}

// Dots <v_k|x> over this block's chunk for k in [k0, k0 + NK), written as partials.  With
// h != nullptr the chunk is first updated in place, x <- x - sum_u h_u v_{ju + u} over u < nu, and
// ||x||^2 of the updated chunk is returned (this happens in the group k0 = 0 only).  NK is the exact
// count: predicated-off FP64 instructions would still take issue slots of the slow FP64 pipe.
template <int NK>
__device__ double chunk_dots_n(const cplx* __restrict__ V, cplx* __restrict__ w, int64_t n, int ju, int nu, int k0,
                               int64_t lo, int64_t hi, const double2* h, double2* part, double* sh, double2* red8) {
    double2 acc[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) acc[k] = make_double2(0.0, 0.0);
    double nn = 0.0;
    const cplx* __restrict__ Vk = V + (int64_t)k0 * n;
    for (int64_t i = lo + threadIdx.x; i < hi; i += OB) {
        double2 x = w[i];
        if (h != nullptr && k0 == 0) {
            for (int k = 0; k < nu; ++k) {
                const double2 v = V[(int64_t)(ju + k) * n + i];
                x.x = fma(-h[k].x, v.x, fma(h[k].y, v.y, x.x));
                x.y = fma(-h[k].x, v.y, fma(-h[k].y, v.x, x.y));
            }
            w[i] = x;
            nn = fma(x.x, x.x, fma(x.y, x.y, nn));
        }
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const double2 v = Vk[(int64_t)k * n + i];   // acc += conj(v) x
            acc[k].x = fma(v.x, x.x, fma(v.y, x.y, acc[k].x));
            acc[k].y = fma(v.x, x.y, fma(-v.y, x.x, acc[k].y));
        }
    }
    block_sum<NK>(acc, sh, red8);
    if (threadIdx.x < NK) part[(int64_t)(k0 + threadIdx.x) * gridDim.x + blockIdx.x] = red8[threadIdx.x];
    return nn;
}

// FP32 value of a double by truncating its mantissa to 23 bits, on the integer pipe (conversions and FP64
// arithmetic share this GPU's narrow FP64 pipe); |x| below 2^-126 gives 0.  Relative error <= 2^-23.
__device__ __forceinline__ float f32_trunc(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), ex = (hi >> 20) & 0x7FFu;
    const unsigned mant = ((hi & 0xFFFFFu) << 3) | ((unsigned)b >> 29);
    return ex <= 896u ? 0.f : __uint_as_float((hi & 0x80000000u) | ((ex - 896u) << 23) | mant);
}

// First-pass dots <v_k|w> over this block's chunk in FP32 (k in [k0, k0 + NK)), written as FP64
// partials.  The second pass (FP64, chunk_dots_n with h) removes what this pass leaves along V to FP64
// accuracy, and alpha is the sum of both passes' coefficients, so only the first pass's FP64 work goes.
template <int NK>
__device__ void chunk_dots_f32_n(const cplx* __restrict__ V, const cplx* __restrict__ w, int64_t n, int k0, int64_t lo,
                                 int64_t hi, double2* part, double* sh, double2* red8) {
    float2 fa[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) fa[k] = make_float2(0.f, 0.f);
    const cplx* __restrict__ Vk = V + (int64_t)k0 * n;
    for (int64_t i = lo + threadIdx.x; i < hi; i += OB) {
        const double2 x = w[i];
        const float xr = f32_trunc(x.x), xi = f32_trunc(x.y);
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const double2 v = Vk[(int64_t)k * n + i];   // acc += conj(v) x
            const float vr = f32_trunc(v.x), vi = f32_trunc(v.y);
            fa[k].x = fmaf(vr, xr, fmaf(vi, xi, fa[k].x));
            fa[k].y = fmaf(vr, xi, fmaf(-vi, xr, fa[k].y));
        }
    }
    double2 acc[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) acc[k] = make_double2((double)fa[k].x, (double)fa[k].y);
    block_sum<NK>(acc, sh, red8);
    if (threadIdx.x < NK) part[(int64_t)(k0 + threadIdx.x) * gridDim.x + blockIdx.x] = red8[threadIdx.x];
}

__device__ void chunk_dots_f32(const cplx* __restrict__ V, const cplx* __restrict__ w, int64_t n, int nv, int k0,
                               int64_t lo, int64_t hi, double2* part, double* sh, double2* red8) {
    switch (min(8, nv - k0)) {
        case 1: return chunk_dots_f32_n<1>(V, w, n, k0, lo, hi, part, sh, red8);
        case 2: return chunk_dots_f32_n<2>(V, w, n, k0, lo, hi, part, sh, red8);
        case 3: return chunk_dots_f32_n<3>(V, w, n, k0, lo, hi, part, sh, red8);
        case 4: return chunk_dots_f32_n<4>(V, w, n, k0, lo, hi, part, sh, red8);
        case 5: return chunk_dots_f32_n<5>(V, w, n, k0, lo, hi, part, sh, red8);
        case 6: return chunk_dots_f32_n<6>(V, w, n, k0, lo, hi, part, sh, red8);
        case 7: return chunk_dots_f32_n<7>(V, w, n, k0, lo, hi, part, sh, red8);
        default: return chunk_dots_f32_n<8>(V, w, n, k0, lo, hi, part, sh, red8);
    }
}

__device__ double chunk_dots(const cplx* __restrict__ V, cplx* __restrict__ w, int64_t n, int nv, int ju, int nu, int k0,
                             int64_t lo, int64_t hi, const double2* h, double2* part, double* sh, double2* red8) {
    switch (min(8, nv - k0)) {
        case 1: return chunk_dots_n<1>(V, w, n, ju, nu, k0, lo, hi, h, part, sh, red8);
        case 2: return chunk_dots_n<2>(V, w, n, ju, nu, k0, lo, hi, h, part, sh, red8);
        case 3: return chunk_dots_n<3>(V, w, n, ju, nu, k0, lo, hi, h, part, sh, red8);
        case 4: return chunk_dots_n<4>(V, w, n, ju, nu, k0, lo, hi, h, part, sh, red8);
        case 5: return chunk_dots_n<5>(V, w, n, ju, nu, k0, lo, hi, h, part, sh, red8);
        case 6: return chunk_dots_n<6>(V, w, n, ju, nu, k0, lo, hi, h, part, sh, red8);
        case 7: return chunk_dots_n<7>(V, w, n, ju, nu, k0, lo, hi, h, part, sh, red8);
        default: return chunk_dots_n<8>(V, w, n, ju, nu, k0, lo, hi, h, part, sh, red8);
    }
}

template <bool SEG>
__global__ void __launch_bounds__(OB) k_lanczos_orth_t(OrthArgs a) {
    pdl_enter();
    // one problem: the whole grid stops together.  Segments: a stopped segment's blocks stay for the grid
    // barriers and do nothing else.
    int sg = 0, b0 = 0, b1 = (int)gridDim.x;
    int64_t lo, hi;
    if (SEG) {
        sg = a.seg.cta_seg[blockIdx.x];
        b0 = a.seg.seg_cta0[sg];
        b1 = a.seg.seg_cta0[sg + 1];
        lo = a.seg.cta_lo[blockIdx.x];
        hi = a.seg.cta_hi[blockIdx.x];
    } else {
        const int64_t ch = (a.n + gridDim.x - 1) / gridDim.x;
        lo = min(a.n, (int64_t)blockIdx.x * ch);
        hi = min(a.n, lo + ch);
    }
    double* tri = a.tri + (SEG ? (int64_t)sg * kTriStride : 0);
    int* flags = a.flags + (SEG ? sg * kFlagStride : 0);
    const bool active = a.j < flags[0];   // uniform per segment: the flag only changes after the last barrier
    if (!SEG && !active) return;
    __shared__ double sh[(OB / 32) * 16];
    __shared__ double2 red8[8];
    __shared__ double2 h[33];
    __shared__ double alpha1;   // the first pass's coefficient of v_j (alpha = pass 1 + pass 2)
    // (A) first-pass dots (FP32) with v_{j-1} and v_j only: H v_j has components above rounding along
    // these two alone (the three-term recurrence), so the first pass skips the older vectors
    const int j0 = a.j > 0 ? a.j - 1 : 0, na = a.j - j0 + 1;
    if (active) chunk_dots_f32(a.V + (int64_t)j0 * a.n, a.w, a.n, na, 0, lo, hi, a.partA, sh, red8);
    grid_barrier(a.bar, a.status);
    // (B) w' = w - h1_{j-1} v_{j-1} - h1_j v_j, second-pass dots with every v_k (FP64), ||w'||^2
    double nn = 0.0;
    if (active) {
        sum_partials(a.partA, na, h, b0, b1);
        if (threadIdx.x == 0) alpha1 = h[na - 1].x;
        for (int k0 = 0; k0 < a.nv; k0 += 8) {
            nn += chunk_dots(a.V, a.w, a.n, a.nv, j0, na, k0, lo, hi, h, a.partB, sh, red8);
            __syncthreads();   // h is read by every thread of the first group
        }
        nn = block_sum1(nn, sh);
        if (threadIdx.x == 0) a.partB[(int64_t)a.nv * gridDim.x + blockIdx.x] = make_double2(nn, 0.0);
    }
    grid_barrier(a.bar, a.status);
    if (!active) return;
    // (C) beta, stop test, v_{j+1} = (w' - sum h2_k v_k) / beta; the scalars by one thread (FP64
    // instructions of the other warps would only repeat them on the slow FP64 pipe)
    sum_partials(a.partB, a.nv + 1, h, b0, b1);
    __shared__ double sc[2];
    if (threadIdx.x == 0) {
        double b2 = h[a.nv].x;
        for (int k = 0; k < a.nv; ++k) b2 -= h[k].x * h[k].x + h[k].y * h[k].y;
        const double bt = sqrt(fmax(b2, 0.0));
        const double alpha = alpha1 + h[a.j].x;
        if (blockIdx.x == b0) tri[T_ALPHA + a.j] = alpha;
        const bool st = (a.j == a.nk - 1) || (bt <= a.tol * fmax(1.0, fabs(alpha)));
        sc[0] = bt;
        sc[1] = st ? 0.0 : 1.0 / bt;
    }
    __syncthreads();
    const double beta = sc[0];
    const bool stop = sc[1] == 0.0;
    if (stop) {
        if (blockIdx.x == b0 && threadIdx.x == 0) {
            tri[T_BETA + a.j] = beta;
            tri[T_RESID] = beta;
            flags[0] = a.j + 1;   // read by later kernels only (every block is past its check)
        }
        return;
    }
    if (blockIdx.x == b0 && threadIdx.x == 0) tri[T_BETA + a.j] = beta;
    const double inv = sc[1];
    cplx* vnext = const_cast<cplx*>(a.V) + (int64_t)(a.j + 1) * a.n;
    for (int64_t i = lo + threadIdx.x; i < hi; i += OB) {
        double2 x = a.w[i];
        for (int k = 0; k < a.nv; ++k) {
            const double2 v = a.V[(int64_t)k * a.n + i];
            x.x = fma(-h[k].x, v.x, fma(h[k].y, v.y, x.x));
            x.y = fma(-h[k].x, v.y, fma(-h[k].y, v.x, x.y));
        }
        vnext[i] = make_double2(x.x * inv, x.y * inv);
    }
}

// Taylor terms for a substep with ||T h|| <= xs <= 2: the smallest K (per bucket of xs) whose remainder
// bound xs^{K+1} / (K+1)! is below 1e-17.
__device__ __forceinline__ int taylor_terms(double xs) {
    return xs <= 0.25 ? 12 : xs <= 0.5 ? 15 : xs <= 0.75 ? 17 : xs <= 1.0 ? 18 : xs <= 1.25 ? 20 : xs <= 1.5 ? 21
         : xs <= 1.75 ? 23 : 24;
}

struct Times { double t[16]; };

// Order key of a time t >= 0: unsigned comparison of the bits is numeric comparison (-0 taken as +0).
__device__ __forceinline__ unsigned long long time_key(double v) {
    return (unsigned long long)__double_as_longlong(v == 0.0 ? 0.0 : v);
}

// 1/k for the Taylor terms (k <= 24), correctly rounded at compile time.
__constant__ double kInvK[25] = {0.0, 1.0 / 1, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8,
                                 1.0 / 9, 1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16,
                                 1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24};

// c_x = beta0 e^{-i T t_x} e_0 for the Lanczos tridiagonal T (alpha, beta), the quantity of
// Eq. lanczosevolution (there written through T = S^dag D S).  GB300 has little FP64 throughput per
// SM, and a Jacobi diagonalisation in one warp spends thousands of dependent FP64 instructions, so
// the vector is advanced directly: one lane per component, (T u)_l from the neighbours by shuffles,
// Taylor series on substeps h with ||T h|| <= nu |h| <= 2 (nu the Gershgorin bound), 12-24 terms
// chosen so that the remainder (nu |h|)^{K+1} / (K+1)! stays below 1e-17.  Targets are reached in
// order of time from t = 0, each from the previous one.  The Krylov error estimate is
// beta_n beta0 |[e^{-i T t_max} e_0]_{n-1}| (t_max the largest target time).
__global__ void __launch_bounds__(32) k_tridiag_exp(double* __restrict__ tri, const int* __restrict__ flags,
                                                     Times times, int n_v, cplx* __restrict__ coef) {
    pdl_enter();
    // one block per segment in segmented mode (a single block otherwise)
    tri += (int64_t)blockIdx.x * kTriStride;
    flags += blockIdx.x * kFlagStride;
    coef += (int64_t)blockIdx.x * kCoefStride;
    __shared__ int order[16];
    const int l = threadIdx.x;
    const int n = flags[0];
    const double b0 = tri[T_BETA0];
    for (int x = 0; x < n_v; ++x) coef[x * 32 + l] = make_double2(0.0, 0.0);
    if (n <= 0) {
        if (l == 0) tri[T_ERR] = 0.0;
        return;
    }
    const double al = l < n ? tri[T_ALPHA + l] : 0.0;
    const double bl = l < n - 1 ? tri[T_BETA + l] : 0.0;   // couples l and l + 1
    double bm = __shfl_up_sync(0xffffffffu, bl, 1);        // couples l - 1 and l
    if (l == 0) bm = 0.0;
    double nu = fabs(al) + fabs(bl) + fabs(bm);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nu = fmax(nu, __shfl_xor_sync(0xffffffffu, nu, o));
    if (l == 0) {   // targets by increasing time
        unsigned long long key[16];
        for (int x = 0; x < n_v; ++x) { key[x] = time_key(times.t[x]); order[x] = x; }
        for (int x = 1; x < n_v; ++x)
            for (int y = x; y > 0 && key[order[y - 1]] > key[order[y]]; --y) { const int t = order[y]; order[y] = order[y - 1]; order[y - 1] = t; }
    }
    __syncwarp();
    int xmax = 0;
    double tmax = 0.0;
    for (int x = 0; x < n_v; ++x)
        if (times.t[x] > tmax) { tmax = times.t[x]; xmax = x; }
    // t_x >= 0 (checked by the entry point): each target from the previous one in time order
    double2 u0 = make_double2(l == 0 ? 1.0 : 0.0, 0.0);   // e^{-i T t_prev} e_0
    double tprev = 0.0;
    for (int m = 0; m < n_v; ++m) {
        const int x = order[m];
        const double dt = times.t[x] - tprev;
        const double span = nu * dt;
        const int S = span > 0.0 ? (int)ceil(0.5 * span) : 0;
        if (S > 0) {
            const double h = dt / S, xs = nu * h;
            const int K = taylor_terms(xs);
            for (int st = 0; st < S; ++st) {
                double2 u = u0, sum = u0;
                for (int k = 1; k <= K; ++k) {
                    const double lx = __shfl_up_sync(0xffffffffu, u.x, 1), ly = __shfl_up_sync(0xffffffffu, u.y, 1);
                    const double rx = __shfl_down_sync(0xffffffffu, u.x, 1), ry = __shfl_down_sync(0xffffffffu, u.y, 1);
                    const double tx = fma(bl, rx, fma(bm, lx, al * u.x));   // (T u)_l; bm = 0 on lane 0,
                    const double ty = fma(bl, ry, fma(bm, ly, al * u.y));   // bl = 0 from lane n - 1 on
                    const double f = h * kInvK[k];
                    u = make_double2(f * ty, -f * tx);                      // (-i h / k) T u
                    sum.x += u.x; sum.y += u.y;
                }
                u0 = sum;
            }
        }
        tprev = times.t[x];
        if (l < n) coef[x * 32 + l] = make_double2(b0 * u0.x, b0 * u0.y);
        if (x == xmax && l == n - 1) tri[T_ERR] = tri[T_RESID] * b0 * sqrt(u0.x * u0.x + u0.y * u0.y);
    }
}

// Targets at equally spaced times m dt (m = 0 .. n_v - 1, target order[m] at m dt): the same c_x as
// k_tridiag_exp, with the chain of dependent Taylor terms one time step long instead of n_v - 1.  Block c
// forms column c of the step exponential E = e^{-i T dt} (the Taylor substeps of k_tridiag_exp from e_c,
// lane l = row l); the last block to finish (ticket) takes u_0 = e_0, u_m = E u_{m-1}.
struct StepTimes { double dt; int n_v, xmax; int order[16]; };
__global__ void __launch_bounds__(32) k_tridiag_exp_eq(double* __restrict__ tri, const int* __restrict__ flags,
                                                        StepTimes st, cplx* __restrict__ coef, cplx* __restrict__ mexp,
                                                        unsigned* __restrict__ ticket) {
    pdl_enter();
    const int l = threadIdx.x, c = blockIdx.x;
    const int n = flags[0];
    if (c < n) {
        const double al = l < n ? tri[T_ALPHA + l] : 0.0;
        const double bl = l < n - 1 ? tri[T_BETA + l] : 0.0;   // couples l and l + 1
        double bm = __shfl_up_sync(0xffffffffu, bl, 1);        // couples l - 1 and l
        if (l == 0) bm = 0.0;
        double nu = fabs(al) + fabs(bl) + fabs(bm);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nu = fmax(nu, __shfl_xor_sync(0xffffffffu, nu, o));
        double2 u0 = make_double2(l == c ? 1.0 : 0.0, 0.0);
        const double span = nu * st.dt;
        const int S = span > 0.0 ? (int)ceil(0.5 * span) : 0;
        if (S > 0) {
            const double h = st.dt / S, xs = nu * h;
            const int K = taylor_terms(xs);
            for (int sb = 0; sb < S; ++sb) {
                double2 u = u0, sum = u0;
                for (int k = 1; k <= K; ++k) {
                    const double lx = __shfl_up_sync(0xffffffffu, u.x, 1), ly = __shfl_up_sync(0xffffffffu, u.y, 1);
                    const double rx = __shfl_down_sync(0xffffffffu, u.x, 1), ry = __shfl_down_sync(0xffffffffu, u.y, 1);
                    const double tx = fma(bl, rx, fma(bm, lx, al * u.x));
                    const double ty = fma(bl, ry, fma(bm, ly, al * u.y));
                    const double f = h * kInvK[k];
                    u = make_double2(f * ty, -f * tx);                      // (-i h / k) T u
                    sum.x += u.x; sum.y += u.y;
                }
                u0 = sum;
            }
        }
        mexp[c * 32 + l] = u0;
    }
    __threadfence();
    unsigned tk = 0;
    if (l == 0) tk = atomicAdd(ticket, 1u);
    tk = __shfl_sync(0xffffffffu, tk, 0);
    if (tk != gridDim.x - 1) return;   // not the last block
    __threadfence();
    if (l == 0) *ticket = 0u;          // every block has taken its ticket: ready for the next launch
    const double b0 = tri[T_BETA0];
    for (int x = 0; x < st.n_v; ++x) coef[x * 32 + l] = make_double2(0.0, 0.0);
    if (n <= 0) {
        if (l == 0) tri[T_ERR] = 0.0;
        return;
    }
    double2 u = make_double2(l == 0 ? 1.0 : 0.0, 0.0);
    for (int m = 0; m < st.n_v; ++m) {
        if (m > 0) {   // u <- E u, two partial sums
            double2 a0 = make_double2(0.0, 0.0), a1 = make_double2(0.0, 0.0);
            for (int cc = 0; cc < n; cc += 2) {   // lanes >= n hold u = 0, so column n (if n is odd) adds 0
                const double ux = __shfl_sync(0xffffffffu, u.x, cc), uy = __shfl_sync(0xffffffffu, u.y, cc);
                const double vx = __shfl_sync(0xffffffffu, u.x, cc + 1), vy = __shfl_sync(0xffffffffu, u.y, cc + 1);
                const double2 e = __ldcg(mexp + cc * 32 + l);
                const double2 f = cc + 1 < n ? __ldcg(mexp + (cc + 1) * 32 + l) : make_double2(0.0, 0.0);
                a0.x = fma(e.x, ux, fma(-e.y, uy, a0.x));
                a0.y = fma(e.x, uy, fma(e.y, ux, a0.y));
                a1.x = fma(f.x, vx, fma(-f.y, vy, a1.x));
                a1.y = fma(f.x, vy, fma(f.y, vx, a1.y));
            }
            u = make_double2(a0.x + a1.x, a0.y + a1.y);
        }
        const int x = st.order[m];
        if (l < n) coef[x * 32 + l] = make_double2(b0 * u.x, b0 * u.y);
        if (x == st.xmax && l == n - 1) tri[T_ERR] = tri[T_RESID] * b0 * sqrt(u.x * u.x + u.y * u.y);
    }
}

// Lowest eigenpair of the Lanczos tridiagonal T (ground-state targeting, Sec. II.B): one thread, FP64.
// The eigenvalue by bisection on the Sturm count (number of eigenvalues below x from the signs of the
// LDL^T pivots of T - x), then the eigenvector by inverse iteration (three tridiagonal solves with the
// shifted matrix, pivots kept away from zero); coef[0][k] = x_k (normalised, real), tri[T_EMIN] = lambda.
__global__ void __launch_bounds__(32) k_tridiag_min(double* __restrict__ tri, const int* __restrict__ flags,
                                                     cplx* __restrict__ coef) {
    pdl_enter();
    if (threadIdx.x != 0) return;
    const int n = flags[0];
    for (int k = 0; k < 32; ++k) coef[k] = make_double2(0.0, 0.0);
    if (n <= 0) { tri[T_EMIN] = 0.0; return; }
    const double* al = tri + T_ALPHA;
    const double* be = tri + T_BETA;   // be[k] couples k and k + 1
    double lo = 1e300, hi = -1e300;
    for (int k = 0; k < n; ++k) {
        const double r = (k > 0 ? fabs(be[k - 1]) : 0.0) + (k + 1 < n ? fabs(be[k]) : 0.0);
        lo = fmin(lo, al[k] - r);
        hi = fmax(hi, al[k] + r);
    }
    const double tiny = 1e-300;
    for (int it = 0; it < 200 && hi - lo > 4e-16 * fmax(fabs(lo), fabs(hi)) + 1e-300; ++it) {
        const double x = 0.5 * (lo + hi);
        int cnt = 0;
        double q = al[0] - x;
        cnt += q < 0.0;
        for (int k = 1; k < n; ++k) {
            if (q == 0.0) q = tiny;
            q = al[k] - x - be[k - 1] * be[k - 1] / q;
            cnt += q < 0.0;
        }
        if (cnt >= 1) hi = x;
        else lo = x;
    }
    const double lam = 0.5 * (lo + hi);
    // a pivot that vanishes (lam an exact eigenvalue, e.g. n = 1 when the start vector is already an
    // eigenvector) is replaced by eps ||T||; each solve is rescaled by its largest entry before the norm
    const double pmin = 2.2e-16 * fmax(fmax(fabs(lo), fabs(hi)), 1e-300);
    double v[32], dg[32], up[32];
    for (int k = 0; k < n; ++k) v[k] = 1.0;
    for (int r = 0; r < 3; ++r) {   // (T - lam) y = v by elimination down the band, then back substitution
        for (int k = 0; k < n; ++k) { dg[k] = al[k] - lam; up[k] = k + 1 < n ? be[k] : 0.0; }
        for (int k = 1; k < n; ++k) {
            if (fabs(dg[k - 1]) < pmin) dg[k - 1] = dg[k - 1] < 0.0 ? -pmin : pmin;
            const double m = be[k - 1] / dg[k - 1];
            dg[k] -= m * up[k - 1];
            v[k] -= m * v[k - 1];
        }
        if (fabs(dg[n - 1]) < pmin) dg[n - 1] = dg[n - 1] < 0.0 ? -pmin : pmin;
        v[n - 1] /= dg[n - 1];
        for (int k = n - 2; k >= 0; --k) v[k] = (v[k] - up[k] * v[k + 1]) / dg[k];
        double mx = 0.0;
        for (int k = 0; k < n; ++k) mx = fmax(mx, fabs(v[k]));
        double nn = 0.0;
        for (int k = 0; k < n; ++k) { v[k] /= mx; nn += v[k] * v[k]; }
        const double inv = 1.0 / sqrt(nn);
        for (int k = 0; k < n; ++k) v[k] *= inv;
    }
    for (int k = 0; k < n; ++k) coef[k] = make_double2(v[k], 0.0);
    tri[T_EMIN] = lam;
}

struct TargetPtrs { cplx* p[16]; };
struct CombineList { cplx* p[8]; int row[8]; };   // targets of one combine launch and their coefficient rows

// targets p[x][i] = sum_k coef[row[x]][k] v_k[i] for x < NX: one pass over V.  NX is exact (no
// predicated FP64 work for absent targets).
template <int NX>
__global__ void __launch_bounds__(256) k_combine(const cplx* __restrict__ V, int64_t n, const int* __restrict__ flags,
                                                  const cplx* __restrict__ coef, CombineList tg) {
    pdl_enter();
    __shared__ double2 cf[NX][32];
    const int nu = flags[0];
    for (int e = threadIdx.x; e < NX * 32; e += blockDim.x) cf[e / 32][e % 32] = coef[tg.row[e / 32] * 32 + e % 32];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 acc[NX];
#pragma unroll
        for (int x = 0; x < NX; ++x) acc[x] = make_double2(0.0, 0.0);
        for (int k = 0; k < nu; ++k) {
            const double2 v = V[(int64_t)k * n + i];
#pragma unroll
            for (int x = 0; x < NX; ++x) {
                const double2 c = cf[x][k];
                acc[x].x = fma(c.x, v.x, fma(-c.y, v.y, acc[x].x));
                acc[x].y = fma(c.x, v.y, fma(c.y, v.x, acc[x].y));
            }
        }
#pragma unroll
        for (int x = 0; x < NX; ++x) tg.p[x][i] = acc[x];
    }
}

// The targets listed in rows (coefficient row of each), eight per launch; returns the launch count.
int launch_combine(const cplx* V, int64_t n, const int* flags, const cplx* coef, const std::vector<int>& rows,
                   const TargetPtrs& tg, int grid, cudaStream_t s) {
    const int cnt = (int)rows.size();
    int launches = 0;
    for (int x0 = 0; x0 < cnt; x0 += 8) {
        CombineList t{};
        for (int x = x0; x < std::min(cnt, x0 + 8); ++x) { t.p[x - x0] = tg.p[rows[x]]; t.row[x - x0] = rows[x]; }
        switch (std::min(8, cnt - x0)) {
            case 1: launch_pdl(k_combine<1>, grid, 256, 0, s, V, n, flags, coef, t); break;
            case 2: launch_pdl(k_combine<2>, grid, 256, 0, s, V, n, flags, coef, t); break;
            case 3: launch_pdl(k_combine<3>, grid, 256, 0, s, V, n, flags, coef, t); break;
            case 4: launch_pdl(k_combine<4>, grid, 256, 0, s, V, n, flags, coef, t); break;
            case 5: launch_pdl(k_combine<5>, grid, 256, 0, s, V, n, flags, coef, t); break;
            case 6: launch_pdl(k_combine<6>, grid, 256, 0, s, V, n, flags, coef, t); break;
            case 7: launch_pdl(k_combine<7>, grid, 256, 0, s, V, n, flags, coef, t); break;
            default: launch_pdl(k_combine<8>, grid, 256, 0, s, V, n, flags, coef, t); break;
        }
        ++launches;
    }
    return launches;
}

// ---- segmented mode: the start vector's norm, v_0 and the targets per segment --------------------
__global__ void __launch_bounds__(NT) k_norm2_seg(const cplx* __restrict__ x, SegTab tb, double2* __restrict__ part) {
    pdl_enter();
    const int64_t lo = tb.cta_lo[blockIdx.x], hi = tb.cta_hi[blockIdx.x];
    double s = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += NT) { const double2 v = x[i]; s += v.x * v.x + v.y * v.y; }
    const double2 t = block_sum(make_double2(s, 0.0));
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) k_init_v0_seg(const cplx* __restrict__ phi, SegTab tb, const double2* __restrict__ part,
                                                    cplx* __restrict__ v0, double* __restrict__ tri, int* __restrict__ flags,
                                                    int nk) {
    pdl_enter();
    __shared__ double b0s;
    const int sg = tb.cta_seg[blockIdx.x], c0 = tb.seg_cta0[sg], c1 = tb.seg_cta0[sg + 1];
    if (threadIdx.x < 32) {   // the segment's partials in a fixed order
        double t = 0.0;
        for (int b = c0 + (int)threadIdx.x; b < c1; b += 32) t += part[b].x;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) b0s = sqrt(t);
    }
    __syncthreads();
    const double b0 = b0s, inv = b0 > 0.0 ? 1.0 / b0 : 0.0;
    const int64_t lo = tb.cta_lo[blockIdx.x], hi = tb.cta_hi[blockIdx.x];
    for (int64_t i = lo + threadIdx.x; i < hi; i += NT) { const double2 v = phi[i]; v0[i] = make_double2(v.x * inv, v.y * inv); }
    if ((int)blockIdx.x == c0 && threadIdx.x == 0) {
        tri[(int64_t)sg * kTriStride + T_BETA0] = b0;
        tri[(int64_t)sg * kTriStride + T_RESID] = 0.0;
        flags[sg * kFlagStride] = b0 > 0.0 ? nk : 0;
    }
}

// targets[x] over each block's range with its segment's coefficients (one pass over V)
template <int NX>
__global__ void __launch_bounds__(256) k_combine_seg(const cplx* __restrict__ V, int64_t n, SegTab tb,
                                                     const int* __restrict__ flags, const cplx* __restrict__ coef, int x0,
                                                     TargetPtrs tg) {
    pdl_enter();
    __shared__ double2 cf[NX][32];
    const int sg = tb.cta_seg[blockIdx.x];
    const int nu = flags[sg * kFlagStride];
    const cplx* cs = coef + (int64_t)sg * kCoefStride;
    for (int e = threadIdx.x; e < NX * 32; e += blockDim.x) cf[e / 32][e % 32] = cs[(x0 + e / 32) * 32 + e % 32];
    __syncthreads();
    const int64_t lo = tb.cta_lo[blockIdx.x], hi = tb.cta_hi[blockIdx.x];
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        double2 acc[NX];
#pragma unroll
        for (int x = 0; x < NX; ++x) acc[x] = make_double2(0.0, 0.0);
        for (int k = 0; k < nu; ++k) {
            const double2 v = V[(int64_t)k * n + i];
#pragma unroll
            for (int x = 0; x < NX; ++x) {
                const double2 c = cf[x][k];
                acc[x].x = fma(c.x, v.x, fma(-c.y, v.y, acc[x].x));
                acc[x].y = fma(c.x, v.y, fma(c.y, v.x, acc[x].y));
            }
        }
#pragma unroll
        for (int x = 0; x < NX; ++x) tg.p[x][i] = acc[x];
    }
}

cudaError_t launch_combine_seg(const cplx* V, int64_t n, const SegTab& tb, int grid, const int* flags, const cplx* coef,
                               int n_v, const TargetPtrs& tg, cudaStream_t s) {
    for (int x0 = 0; x0 < n_v; x0 += 8) {
        TargetPtrs t{};
        for (int x = x0; x < n_v; ++x) t.p[x - x0] = tg.p[x];
        switch (std::min(8, n_v - x0)) {
            case 1: launch_pdl(k_combine_seg<1>, grid, 256, 0, s, V, n, tb, flags, coef, x0, t); break;
            case 2: launch_pdl(k_combine_seg<2>, grid, 256, 0, s, V, n, tb, flags, coef, x0, t); break;
            case 3: launch_pdl(k_combine_seg<3>, grid, 256, 0, s, V, n, tb, flags, coef, x0, t); break;
            case 4: launch_pdl(k_combine_seg<4>, grid, 256, 0, s, V, n, tb, flags, coef, x0, t); break;
            case 5: launch_pdl(k_combine_seg<5>, grid, 256, 0, s, V, n, tb, flags, coef, x0, t); break;
            case 6: launch_pdl(k_combine_seg<6>, grid, 256, 0, s, V, n, tb, flags, coef, x0, t); break;
            case 7: launch_pdl(k_combine_seg<7>, grid, 256, 0, s, V, n, tb, flags, coef, x0, t); break;
            default: launch_pdl(k_combine_seg<8>, grid, 256, 0, s, V, n, tb, flags, coef, x0, t); break;
        }
    }
    return cudaGetLastError();
}

__global__ void __launch_bounds__(NT) k_dot2(const cplx* __restrict__ x, const cplx* __restrict__ y, int64_t n,
                                              double2* __restrict__ part) {
    pdl_enter();
    int64_t lo, hi;
    chunk_of(n, lo, hi);
    double2 s = make_double2(0.0, 0.0);
    double nn = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += NT) {
        const double2 a = x[i];
        const double2 p = cdotc(a, y[i]);
        s.x += p.x; s.y += p.y;
        nn += a.x * a.x + a.y * a.y;
    }
    double2 t = block_sum(s);
    double2 u = block_sum(make_double2(nn, 0.0));
    if (threadIdx.x == 0) { part[blockIdx.x] = t; part[NB + blockIdx.x] = u; }
}

__global__ void __launch_bounds__(NT) k_dot_final(const double2* __restrict__ part, cplx* __restrict__ out, int normalise) {
    pdl_enter();
    __shared__ double2 h[2];
    reduce_coeffs(part, 2, h);
    if (threadIdx.x == 0) {
        double2 v = h[0];
        if (normalise) {
            const double d = h[1].x > 0.0 ? 1.0 / h[1].x : 0.0;
            v.x *= d; v.y *= d;
        }
        *out = v;
    }
}

int ensure_work(tdmrg_ctx* c, int a, int b, int nk, int64_t n, KrylovWork** out) {
    auto key = std::make_pair(a * 4096 + b, nk);
    auto it = c->krylov.find(key);
    if (it != c->krylov.end() && it->second.n == n) { *out = &it->second; return TDMRG_OK; }
    KrylovWork k;
    k.n = n;
    k.nk = nk;
    int rc = dev_alloc(c, (void**)&k.V, (size_t)(nk + 1) * n * sizeof(cplx), "Krylov vectors");
    if (!rc) rc = dev_alloc(c, (void**)&k.w, (size_t)n * sizeof(cplx), "Krylov residual");
    if (!rc) rc = dev_alloc(c, (void**)&k.partA, 64 * kRedBlocks * sizeof(double2), "Krylov partials");
    if (!rc) rc = dev_alloc(c, (void**)&k.partB, 64 * kRedBlocks * sizeof(double2), "Krylov partials");
    if (!rc) rc = dev_alloc(c, (void**)&k.tri, 128 * sizeof(double), "Krylov tridiagonal");
    if (!rc) rc = dev_alloc(c, (void**)&k.flags, 4 * sizeof(int), "Krylov flags");
    // coefficients [x][k] of 16 targets, then the columns of the step exponential (32 x 32)
    if (!rc) rc = dev_alloc(c, (void**)&k.coef, kCoefWords * sizeof(cplx), "Krylov coefficients");
    // grid barrier counter (word 0), then the ticket of k_tridiag_exp_eq (word 2)
    if (!rc) rc = dev_alloc(c, (void**)&k.bar, kBarWords * sizeof(unsigned), "Krylov grid barrier");
    if (!rc) rc = cuda_check(c, cudaMemset(k.bar, 0, kBarWords * sizeof(unsigned)), "Krylov grid barrier");
    if (!rc) {   // co-resident grid of the fused orthogonalisation: at most one block per SM, at most NB
        int per_sm = 0;
        rc = cuda_check(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lanczos_orth_t<true>, OB, 0), "occupancy");
        const int want = c->orth_per_sm > 0 ? c->orth_per_sm : 1;   // blocks per SM of the fused orthogonalisation
        k.orth_grid = std::max(1, std::min({c->num_sms * std::max(per_sm, 1), c->num_sms * want, NB}));
    }
    if (rc) {
        dev_free(c, k.V, (size_t)(nk + 1) * n * sizeof(cplx));
        dev_free(c, k.w, (size_t)n * sizeof(cplx));
        dev_free(c, k.partA, 64 * kRedBlocks * sizeof(double2));
        dev_free(c, k.partB, 64 * kRedBlocks * sizeof(double2));
        dev_free(c, k.tri, 128 * sizeof(double));
        dev_free(c, k.flags, 4 * sizeof(int));
        dev_free(c, k.coef, kCoefWords * sizeof(cplx));
        dev_free(c, k.bar, kBarWords * sizeof(unsigned));
        return rc;
    }
    c->krylov[key] = k;
    *out = &c->krylov[key];
    return TDMRG_OK;
}

}  // namespace

cudaError_t launch_norm2(const cplx* x, int64_t n, double2* partials, int nblk, cudaStream_t s) {
    (void)nblk;
    launch_pdl(k_norm2, NB, NT, 0, s, x, n, partials);
    return cudaGetLastError();
}

cudaError_t launch_dot_final(const cplx* x, const cplx* y, int64_t n, double2* partials, int nblk, cplx* out,
                             int normalise, cudaStream_t s) {
    (void)nblk;
    launch_pdl(k_dot2, NB, NT, 0, s, x, y, n, partials);
    launch_pdl(k_dot_final, 1, NT, 0, s, partials, out, normalise);
    return cudaGetLastError();
}

// The Lanczos recursion of n_K steps started at phi (Sec. II.A): V, the tridiagonal and the flags in the
// Krylov workspace of (Q, nk).
int lanczos_build(tdmrg_ctx* c, int a, int b, const cplx* phi, int nk, KrylovWork** out) {
    int64_t n = sector_size(c, a, b);
    if (n == 0) return fail(c, TDMRG_ESECTOR, "Lanczos: empty sector");
    Plan* p = nullptr;
    int rc = get_ham_plan(c, a, b, &p);
    if (rc) return rc;
    KrylovWork* k = nullptr;
    rc = ensure_work(c, a, b, nk, n, &k);
    if (rc) return rc;
    *out = k;
    cudaStream_t s = c->stream;
    launch_pdl(k_norm2, NB, NT, 0, s, phi, n, k->partA);
    launch_pdl(k_init_v0, NB, NT, 0, s, phi, n, k->partA, k->V, k->tri, k->flags, nk);
    c->launches += 2;
    for (int j = 0; j < nk; ++j) {
        cplx* vj = k->V + (int64_t)j * n;
        rc = run_plan(c, *p, vj, k->w, k->flags, j);
        if (rc) return rc;
        OrthArgs oa{k->V, k->w, n, j + 1, j, nk, c->opts.breakdown_tol, k->partA, k->partB, k->tri, k->flags,
                    k->bar, c->dstatus};
        void* params[] = {&oa};
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(k->orth_grid);
        cfg.blockDim = dim3(OB);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t le = cudaLaunchKernelExC(&cfg, (const void*)k_lanczos_orth_t<false>, params);
        if (le != cudaSuccess) return cuda_check(c, le, "Lanczos orthogonalisation launch");
        c->launches += 1;
    }
    return TDMRG_OK;
}

int evolve(tdmrg_ctx* c, int a, int b, const cplx* phi, int n_v, const double* t_x, int nk, cplx* const* targets) {
    KrylovWork* k = nullptr;
    int rc = lanczos_build(c, a, b, phi, nk, &k);
    if (rc) return rc;
    const int64_t n = k->n;
    cudaStream_t s = c->stream;
    Times tt{};
    for (int x = 0; x < n_v; ++x) tt.t[x] = t_x[x];
    // equally spaced targets from t = 0 (the TST schedule): one time step's Taylor chain, columns in parallel
    std::vector<int> ord(n_v);
    for (int x = 0; x < n_v; ++x) ord[x] = x;
    std::stable_sort(ord.begin(), ord.end(), [&](int p, int q) { return t_x[p] < t_x[q]; });
    const double tmax = t_x[ord[n_v - 1]];
    bool eq = n_v >= 2 && n_v <= 16 && t_x[ord[0]] == 0.0 && t_x[ord[1]] > 0.0;
    const double dt = eq ? t_x[ord[1]] : 0.0;
    for (int m = 2; m < n_v && eq; ++m) eq = std::fabs(t_x[ord[m]] - m * dt) <= 8.0 * 2.220446049250313e-16 * tmax;
    if (eq) {
        StepTimes st{};
        st.dt = dt; st.n_v = n_v; st.xmax = ord[n_v - 1];
        for (int m = 0; m < n_v; ++m) st.order[m] = ord[m];
        launch_pdl(k_tridiag_exp_eq, k->nk, 32, 0, s, k->tri, k->flags, st, k->coef, k->coef + 16 * 32, k->bar + 2);
    } else {
        launch_pdl(k_tridiag_exp, 1, 32, 0, s, k->tri, k->flags, tt, n_v, k->coef);
    }
    // a target at t = 0 is phi itself: copied (before any target that aliases phi is written), not combined
    std::vector<int> rows;
    for (int x = 0; x < n_v; ++x) {
        if (t_x[x] != 0.0) { rows.push_back(x); continue; }
        if (targets[x] != phi) {
            int rc2 = cuda_check(c, cudaMemcpyAsync(targets[x], phi, (size_t)n * sizeof(cplx), cudaMemcpyDeviceToDevice, s),
                                 "evolve copy");
            if (rc2) return rc2;
        }
    }
    TargetPtrs tg{};
    for (int x = 0; x < n_v; ++x) tg.p[x] = targets[x];
    int grid = (int)std::min<int64_t>((n + 255) / 256, 4L * c->num_sms);
    c->launches += 1 + launch_combine(k->V, n, k->flags, k->coef, rows, tg, grid, s);
    c->last_krylov = k;
    return cuda_check(c, cudaGetLastError(), "evolve launch");
}

// Ground state in sector Q (ground-state targeting, Sec. II.B): `restarts` times, Lanczos with nk steps from
// psi, the lowest eigenvector of T combined in place into psi.
int ground_state(tdmrg_ctx* c, int a, int b, cplx* psi, int nk, int restarts, double* energy) {
    KrylovWork* k = nullptr;
    for (int r = 0; r < restarts; ++r) {
        int rc = lanczos_build(c, a, b, psi, nk, &k);
        if (rc) return rc;
        launch_pdl(k_tridiag_min, 1, 32, 0, c->stream, k->tri, k->flags, k->coef);
        TargetPtrs tg{};
        tg.p[0] = psi;
        const int grid = (int)std::min<int64_t>((k->n + 255) / 256, 4L * c->num_sms);
        launch_combine(k->V, k->n, k->flags, k->coef, std::vector<int>{0}, tg, grid, c->stream);
        c->launches += 2;
        rc = cuda_check(c, cudaGetLastError(), "ground-state launch");
        if (rc) return rc;
    }
    c->last_krylov = k;
    double tri[128];
    int rc = cuda_check(c, cudaMemcpyAsync(tri, k->tri, sizeof(tri), cudaMemcpyDeviceToHost, c->stream), "ground state");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "ground state");
    if (!rc) rc = check_device_status(c);
    if (!rc && energy) *energy = tri[T_EMIN];
    return rc;
}

// Device tables of the segmented mode: the CTA partition (each segment gets CTAs in proportion to its
// length, at least one) and the per-segment Krylov state, allocated with the Krylov workspace.
static int ensure_segments(tdmrg_ctx* c, KrylovWork* k, int nseg, const int64_t* seg_len, SegTab* tb, double** tri,
                           int** flags, cplx** coef, int* grid) {
    const int G = k->orth_grid;
    if (nseg < 1 || nseg > G) return fail(c, TDMRG_EINVAL, "evolve_segments: more segments than co-resident blocks");
    const bool same = k->nseg == nseg && std::equal(k->seg_len.begin(), k->seg_len.end(), seg_len) &&
                      (int)k->seg_len.size() == nseg;
    const size_t b_tri = (size_t)nseg * kTriStride * sizeof(double), b_fl = (size_t)nseg * kFlagStride * sizeof(int);
    const size_t b_co = (size_t)nseg * kCoefStride * sizeof(cplx), b_cs = (size_t)G * sizeof(int);
    const size_t b_lo = (size_t)G * sizeof(int64_t), b_c0 = (size_t)(nseg + 1) * sizeof(int);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t bytes = al(b_tri) + al(b_fl) + al(b_co) + al(b_cs) + 2 * al(b_lo) + al(b_c0);
    unsigned char* m = (unsigned char*)k->segmem;
    if (!same) {
        // partition: CTAs in proportion to the lengths, at least one per segment
        int64_t n = 0;
        for (int s = 0; s < nseg; ++s) n += seg_len[s];
        std::vector<int> cnt(nseg, 1);
        int left = G - nseg;
        for (int s = 0; s < nseg && n > 0; ++s) {
            const int extra = (int)((double)left * (double)seg_len[s] / (double)n);
            cnt[s] += extra;
        }
        int used = 0;
        for (int s = 0; s < nseg; ++s) used += cnt[s];
        for (int s = 0; used < G; s = (s + 1) % nseg) { ++cnt[s]; ++used; }
        std::vector<int> cta_seg, c0(nseg + 1, 0);
        std::vector<int64_t> lo, hi;
        int64_t off = 0;
        for (int s = 0; s < nseg; ++s) {
            c0[s] = (int)cta_seg.size();
            const int64_t ch = (seg_len[s] + cnt[s] - 1) / cnt[s];
            for (int b = 0; b < cnt[s]; ++b) {
                cta_seg.push_back(s);
                lo.push_back(off + std::min(seg_len[s], (int64_t)b * ch));
                hi.push_back(off + std::min(seg_len[s], (int64_t)(b + 1) * ch));
            }
            off += seg_len[s];
        }
        c0[nseg] = (int)cta_seg.size();
        if (k->segmem_bytes < bytes) {
            dev_free(c, k->segmem, k->segmem_bytes);
            k->segmem = nullptr;
            k->segmem_bytes = 0;
            int rc = dev_alloc(c, &k->segmem, bytes, "Krylov segments");
            if (rc) return rc;
            k->segmem_bytes = bytes;
        }
        m = (unsigned char*)k->segmem;
        std::vector<unsigned char> h(al(b_cs) + 2 * al(b_lo) + al(b_c0), 0);
        memcpy(h.data(), cta_seg.data(), b_cs);
        memcpy(h.data() + al(b_cs), lo.data(), b_lo);
        memcpy(h.data() + al(b_cs) + al(b_lo), hi.data(), b_lo);
        memcpy(h.data() + al(b_cs) + 2 * al(b_lo), c0.data(), b_c0);
        int rc = cuda_check(c, cudaMemcpyAsync(m + al(b_tri) + al(b_fl) + al(b_co), h.data(), h.size(), cudaMemcpyHostToDevice,
                                               c->stream), "Krylov segments");
        if (!rc) rc = cuda_check(c, cudaMemsetAsync(m, 0, al(b_tri) + al(b_fl) + al(b_co), c->stream), "Krylov segments");
        if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "Krylov segments");
        if (rc) return rc;
        k->nseg = nseg;
        k->seg_len.assign(seg_len, seg_len + nseg);
    }
    *tri = (double*)m;
    *flags = (int*)(m + al(b_tri));
    *coef = (cplx*)(m + al(b_tri) + al(b_fl));
    unsigned char* t = m + al(b_tri) + al(b_fl) + al(b_co);
    tb->cta_seg = (const int*)t;
    tb->cta_lo = (const int64_t*)(t + al(b_cs));
    tb->cta_hi = (const int64_t*)(t + al(b_cs) + al(b_lo));
    tb->seg_cta0 = (const int*)(t + al(b_cs) + 2 * al(b_lo));
    tb->nseg = nseg;
    *grid = G;
    return TDMRG_OK;
}

// Independent Krylov advances side by side (Sec. II.A, Eq. lanczosevolution for each segment): one H psi
// over the whole vector per Lanczos step (the superblock is a direct sum, so its products never mix
// segments), orthogonalisation, tridiagonal exponentials and targets per segment.
int evolve_segments(tdmrg_ctx* c, int a, int b, const cplx* phi, int nseg, const int64_t* seg_len, int n_v,
                    const double* t_x, int nk, cplx* const* targets) {
    const int64_t n = sector_size(c, a, b);
    if (n == 0) return fail(c, TDMRG_ESECTOR, "evolve_segments: empty sector");
    int64_t tot = 0;
    for (int s = 0; s < nseg; ++s) {
        if (seg_len[s] < 1) return fail(c, TDMRG_EINVAL, "evolve_segments: empty segment");
        tot += seg_len[s];
    }
    if (tot != n) return fail(c, TDMRG_EINVAL, "evolve_segments: the segment lengths do not add up to the sector size");
    Plan* p = nullptr;
    int rc = get_ham_plan(c, a, b, &p);
    if (rc) return rc;
    KrylovWork* k = nullptr;
    rc = ensure_work(c, a, b, nk, n, &k);
    if (rc) return rc;
    SegTab tb{};
    double* tri = nullptr;
    int* flags = nullptr;
    cplx* coef = nullptr;
    int G = 0;
    rc = ensure_segments(c, k, nseg, seg_len, &tb, &tri, &flags, &coef, &G);
    if (rc) return rc;
    cudaStream_t s = c->stream;
    launch_pdl(k_norm2_seg, G, NT, 0, s, phi, tb, k->partA);
    launch_pdl(k_init_v0_seg, G, NT, 0, s, phi, tb, k->partA, k->V, tri, flags, nk);
    c->launches += 2;
    for (int j = 0; j < nk; ++j) {
        cplx* vj = k->V + (int64_t)j * n;
        rc = run_plan(c, *p, vj, k->w, nullptr, 0);   // every segment's product (a stopped one's is ignored)
        if (rc) return rc;
        OrthArgs oa{k->V, k->w, n, j + 1, j, nk, c->opts.breakdown_tol, k->partA, k->partB, tri, flags, k->bar,
                    c->dstatus, tb};
        void* params[] = {&oa};
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(G);
        cfg.blockDim = dim3(OB);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t le = cudaLaunchKernelExC(&cfg, (const void*)k_lanczos_orth_t<true>, params);
        if (le != cudaSuccess) return cuda_check(c, le, "segmented Lanczos launch");
        c->launches += 1;
    }
    Times tt{};
    for (int x = 0; x < n_v; ++x) tt.t[x] = t_x[x];
    launch_pdl(k_tridiag_exp, nseg, 32, 0, s, tri, flags, tt, n_v, coef);
    TargetPtrs tg{};
    for (int x = 0; x < n_v; ++x) tg.p[x] = targets[x];
    launch_combine_seg(k->V, n, tb, G, flags, coef, n_v, tg, s);
    c->launches += 1 + (n_v + 7) / 8;
    return cuda_check(c, cudaGetLastError(), "evolve_segments launch");
}

// Krylov dimension used and error estimate of each segment of the last evolve_segments on (Q, nk).
int segments_info(tdmrg_ctx* c, int a, int b, int nk, int nseg, int* nk_used, double* err) {
    auto it = c->krylov.find(std::make_pair(a * 4096 + b, nk));
    if (it == c->krylov.end() || it->second.nseg != nseg || !it->second.segmem)
        return fail(c, TDMRG_ESTATE, "evolve_segments_info: no segmented evolve with these arguments");
    std::vector<double> tri((size_t)nseg * kTriStride);
    std::vector<int> fl((size_t)nseg * kFlagStride);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const unsigned char* m = (const unsigned char*)it->second.segmem;
    int rc = cuda_check(c, cudaMemcpyAsync(tri.data(), m, tri.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "info");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(fl.data(), m + al(tri.size() * sizeof(double)), fl.size() * sizeof(int),
                                                cudaMemcpyDeviceToHost, c->stream), "info");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "info");
    if (!rc) rc = check_device_status(c);
    if (rc) return rc;
    for (int s = 0; s < nseg; ++s) {
        if (nk_used) nk_used[s] = fl[(size_t)s * kFlagStride];
        if (err) err[s] = tri[(size_t)s * kTriStride + T_ERR];
    }
    return TDMRG_OK;
}

int evolve_info(tdmrg_ctx* c, int* nk_used, double* err, double* alpha, double* beta) {
    KrylovWork* k = c->last_krylov;
    double tri[128];
    int flags[4];
    int rc = cuda_check(c, cudaMemcpyAsync(tri, k->tri, sizeof(tri), cudaMemcpyDeviceToHost, c->stream), "evolve_info");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(flags, k->flags, sizeof(flags), cudaMemcpyDeviceToHost, c->stream), "evolve_info");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "evolve_info sync");
    if (rc) return rc;
    rc = check_device_status(c);
    if (rc) return rc;
    if (nk_used) *nk_used = flags[0];
    if (err) *err = tri[T_ERR];
    for (int j = 0; j < flags[0]; ++j) {
        if (alpha) alpha[j] = tri[T_ALPHA + j];
        if (beta) beta[j] = tri[T_BETA + j];
    }
    return TDMRG_OK;
}

}  // namespace tdmrg
