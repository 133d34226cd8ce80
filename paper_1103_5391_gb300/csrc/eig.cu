// Eigendecomposition of rho_L per left sector (truncation input of Sec. II.B), FP64 accurate.
//
// GB300 runs FP64 at about 1 TFLOP/s chip-wide (~7 GFLOP/s per SM), so an FP64 Jacobi on one SM per
// sector would take milliseconds for the largest sectors.  Instead:
//   1. seed: a cyclic two-sided Jacobi in FP32 per sector (one CTA per sector, parallel round-robin
//      ordering of disjoint rotations), giving eigenvectors X0 accurate to about 1e-6;
//   2. refine: iterative refinement for Hermitian eigenproblems (Ogita & Aishima, 2018), whose work is
//      grouped GEMMs spread over every SM (FP64, except the small correction E^H W in FP32):
//         G = X^H X,  S = X^H (rho X),  lambda_i = Re S_ii / Re G_ii,  R = I - G,
//         E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)   if |lambda_i - lambda_j| > delta,
//         E_ij = R_ij / 2 otherwise (and on the diagonal),  delta = 2 (||S - diag(lambda)|| + ||rho|| ||R||),
//         X <- X (I + E);
//      convergence is quadratic: from the FP32 seed (error ~1e-5) two iterations reach rounding level;
//      up to four more run (decided on the device, launched regardless) while the last correction is
//      above 1e-7, as for near-degenerate pairs that the first iteration treats as a cluster.  If the
//      sixth is still above it (density matrices of DMRG blocks whose spectra span the whole FP64 range in
//      large degenerate multiplets), two last steps only orthonormalise W (E = R / 2 for every pair, a
//      Newton-Schulz step: orthogonality error eps -> ~eps^2 -> rounding), so that the kept states always
//      form an orthonormal basis and the renormalised operators are projections.  At
//      iterations 1 and 3 a sector whose clustered pairs stay coupled is re-seeded instead (FP32 Jacobi
//      on S with a relative criterion, k_jacobi32).  The iterate is kept as W = X^H, so every product
//      is a plain or conjugate-transposed GEMM operand;
//   3. sort each sector's eigenpairs by descending eigenvalue.
// The sectors run in one group, or in two on two streams: the few with the longest Jacobi seeds (the
// seed of a sector runs on one SM, so its cost grows with n, not with the total work) seed and refine on
// a second stream while the others' seeds and refinement fill the rest of the GPU; a cost model picks the
// split (long_sectors).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace tdmrg {
namespace {

constexpr int JT = 1024;  // threads of the FP32 Jacobi CTA (warps over rotation pairs, lanes over rows)
constexpr int kSmemMaxN = 112;   // A and V as float2 in shared memory: 2 * 112 * 113 * 8 B = 198 KB
constexpr int kSmemMaxA = 158;   // A alone in shared memory (158 * 159 * 8 B = 196 KB), V in global memory
constexpr int kJacSmemCap = 225 * 1024;   // dynamic shared memory of the Jacobi CTA at most
constexpr int kMaxEigN = 512;    // largest sector dimension
constexpr int kKChunk = 16;      // K chunk of the refinement GEMMs
constexpr int kRefine = 2;       // refinement iterations always run
constexpr int kOaIters = 6;      // more, each only when the previous correction was not yet small
constexpr int kMaxRefine = 8;    // then, if the last one was still not small, two steps that only orthonormalise W
constexpr float kReseedTol = 1e-7f;    // re-seed rotates (p, q) while |S_pq| > kReseedTol sqrt|S_pp S_qq| ...
constexpr float kReseedFloor = 1e-14f; // ... and |S_pq| > kReseedFloor ||rho||_F
// Refinement iterations that may re-seed a sector instead of updating it.
__host__ __device__ constexpr bool reseed_iter(int it) { return it == 1 || it == 3; }
constexpr double kTolE = 1e-7;   // |E| above this: the next error (~|E|^2) may exceed ~1e-14

struct EigTables {
    const int64_t* off;   // per sector: offset of its n x n block
    const int64_t* eoff;  // per sector: offset of its eigenvalues
    const int64_t* roff;  // per sector: offset of its global rotation record (sectors beyond kSmemMaxN)
    const int* dims;
    const int* big;       // the sectors beyond kSmemMaxN, in table order
};
constexpr int kMaxSweeps = 12;     // Jacobi sweeps at most (the record holds this many)
constexpr int kReplayRows = 8;     // rows of V per CTA of the record replay
constexpr int kReplayThreads = 512;

__device__ __forceinline__ float2 cmf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// Rotation J = [[c, s], [-conj(s), c]] on (p, q) annihilating b = A_pq of the Hermitian 2x2 block
// [[a, b], [conj(b), d]], written without divisions: with x = d - a and r = sqrt(x^2 + 4|b|^2),
// tan = sign(x) 2|b| / (|x| + r) gives c = (|x| + r) w and s = sign(x) 2 b w, w = 1 / sqrt(2 r (|x| + r)).
// A Newton step on 1 / sqrt(c^2 + |s|^2) then makes J unitary to about one ulp, so the hundreds of
// rotations accumulated in V keep it orthonormal to ~1e-6.
__device__ __forceinline__ void rotation32(float a, float d, float2 b, float& c, float2& s) {
    const float x = d - a, ax = fabsf(x);
    const float v = fmaf(x, x, 4.f * fmaf(b.x, b.x, b.y * b.y));
    const float r = v * rsqrtf(v);
    const float w = rsqrtf(2.f * r * (ax + r));
    const float sg = x < 0.f ? -2.f * w : 2.f * w;
    c = (ax + r) * w;
    s = make_float2(sg * b.x, sg * b.y);
    const float f = fmaf(-0.5f, fmaf(c, c, fmaf(s.x, s.x, s.y * s.y)), 1.5f);
    c *= f;
    s.x *= f; s.y *= f;
}

// Round-robin pairing of round `round`: pair i of P / 2 disjoint index pairs (p < q); index P - 1 = n
// is a dummy when n is odd.
__device__ __forceinline__ void rr_pair(int round, int i, int P, int& p, int& q) {
    if (i == 0) { p = P - 1; q = round; }
    else {   // (round + i) and (round - i) mod P - 1, with 0 <= round < P - 1 and 0 < i < P / 2
        p = round + i; if (p >= P - 1) p -= P - 1;
        q = round - i; if (q < 0) q += P - 1;
    }
    if (p > q) { int t = p; p = q; q = t; }
}

__device__ __forceinline__ float2 rot_l(float c, float2 s, float2 x, float2 y) {   // c x - s y
    const float2 t = cmf(s, y);
    return make_float2(c * x.x - t.x, c * x.y - t.y);
}
__device__ __forceinline__ float2 rot_r(float c, float2 s, float2 x, float2 y) {   // s x + c y
    const float2 t = cmf(s, x);
    return make_float2(t.x + c * y.x, t.y + c * y.y);
}

constexpr int JA = 512;   // threads that rotate A (warps 0-15); the other 16 warps accumulate V

// Where a sector's Jacobi keeps its matrices: A and V in shared memory (n <= kSmemMaxN); A in shared
// memory and V in global memory, stored transposed so that the V warps' accesses along a column are
// contiguous (n <= kSmemMaxA); both in global memory (larger n).
enum JacMode { JAC_SMEM = 0, JAC_SMEM_A = 1, JAC_GLOBAL = 2 };
__host__ __device__ inline int jac_mode(int n) { return n <= kSmemMaxN ? JAC_SMEM : n <= kSmemMaxA ? JAC_SMEM_A : JAC_GLOBAL; }

// Sectors whose V is formed afterwards from a global rotation record (V not in shared memory).
__host__ __device__ inline bool jac_recorded(int n) { return n > kSmemMaxN; }

// Rounds of the rotation record that fit in `smem` bytes beside A and V (two buffers of float4 per pair).
__host__ __device__ inline int jac_base_bytes(int n) {
    const int m = jac_mode(n);
    return m == JAC_SMEM ? 16 * n * (n | 1) : m == JAC_SMEM_A ? ((8 * n * (n | 1) + 15) & ~15) : 0;
}
__host__ __device__ inline int jac_chunk(int n, int smem) {
    const int P = n + (n & 1), R = P - 1, npair = P / 2;
    if (npair == 0) return 1;
    const int c = (smem - jac_base_bytes(n)) / (32 * npair);
    return c < R ? c : R;
}

// V <- V J_r for the recorded rounds r0 .. r0 + nr - 1 (V group: warps over pairs, lanes over rows, so a
// warp's accesses to a column of V fall in distinct banks; a V-group barrier separates the rounds).
// Element (k, p) of V is at V[k * rs + p * cs]: row-major in shared memory (rs = ld, cs = 1), transposed
// in global memory (rs = 1, cs = ld), where a warp's accesses along a column are then contiguous.
__device__ __forceinline__ void jacobi_apply_v(float2* V, int n, int rs, int cs, const float4* rec, int nr, int r0) {
    const int P = n + (n & 1), npair = P / 2;
    const int lane = threadIdx.x & 31, vw = (threadIdx.x - JA) >> 5;
    constexpr int NVW = (JT - JA) / 32;
    for (int r = 0; r < nr; ++r) {
        for (int i = vw; i < npair; i += NVW) {
            const float4 ro = rec[r * npair + i];
            if (ro.y == 0.f && ro.z == 0.f) continue;   // identity
            const int p = __float_as_int(ro.w) & 0xffff, q = __float_as_int(ro.w) >> 16;
            const float c = ro.x;
            const float2 s = make_float2(ro.y, ro.z), sc = conjf2(s);
            float2* Vp = V + p * cs;
            float2* Vq = V + q * cs;
            for (int k = lane; k < n; k += 32) {
                const float2 vp = Vp[k * rs], vq = Vq[k * rs];
                Vp[k * rs] = rot_l(c, sc, vp, vq);
                Vq[k * rs] = rot_r(c, s, vp, vq);
            }
        }
        asm volatile("bar.sync 2, %0;" ::"r"(JT - JA) : "memory");
    }
}

// Cyclic two-sided Jacobi on the Hermitian A (n x n, row stride ld), eigenvectors accumulated in
// V, both either in shared or in global memory (the body is inlined once for each so that shared
// accesses compile as such).  Each round: threads of the A group compute the rotations of the round's
// disjoint pairs and record them (with the pair's indices); after a barrier of the A group, each 2 x 2
// block (pair a, pair b <= a) of A is rotated on both sides at once, A <- J^H A J, and written back
// together with its mirror image (plain loads, no triangle addressing).  The V
// group replays the record of the previous chunk of rounds on V meanwhile; record buffers swap at a
// barrier of all threads every `C` rounds.
//
// Criterion: (p, q) is rotated while |A_pq|^2 > lim, lim = thr^2 for the seed, and for the re-seed
// (`rel`) lim = max(kReseedTol^2 |A_pp A_qq|, floor^2), relative to the pair's own diagonal.
__device__ __forceinline__ float jac_lim(bool rel, float thr2, float a, float d) {
    return rel ? fmaxf(kReseedTol * kReseedTol * fabsf(a * d), thr2) : thr2;
}
//
// Record mode (grec != nullptr, used when V does not fit in shared memory): every thread rotates A
// (ja = JT), each rotation is also written to the global record grec (round-major, npair per round) and
// *nrec receives the number of rounds; V is formed afterwards from the record by k_jacobi_replay.
__device__ __forceinline__ int jacobi_sweeps(float2* A, float2* V, int n, int ld, int vrs, int vcs, float thr, bool rel,
                                             float4* rec, int C, int ja, float4* __restrict__ grec, int* nrec) {
    const int tid = threadIdx.x;
    const bool agroup = tid < ja;
    int total = 0;   // rounds recorded before the current chunk
    const float thr2 = thr * thr;
    const int P = n + (n & 1), npair = P / 2, R = P - 1;
    const int warp = tid >> 5, lane = tid & 31;
    int pend = 0, pend_r0 = 0, buf = 0;
    bool done = n <= 1;
    int sweep = 0;
    for (; sweep < 12 && !done; ++sweep) {
        for (int r0 = 0; r0 < R; r0 += C) {
            const int nr = min(C, R - r0);
            const bool last = r0 + nr >= R;
            float4* cur = rec + (size_t)buf * C * npair;
            bool above = false;
            if (agroup) {
                for (int r = 0; r < nr; ++r) {
                    const int round = r0 + r;
                    float4* rr = cur + r * npair;
                    for (int i = tid; i < npair; i += ja) {
                        int p, q;
                        rr_pair(round, i, P, p, q);
                        float c = 1.f;
                        float2 s = make_float2(0.f, 0.f);
                        if (q < n) {
                            const float2 b = A[p * ld + q];
                            const float ap = A[p * ld + p].x, aq = A[q * ld + q].x;
                            if (fmaf(b.x, b.x, b.y * b.y) <= jac_lim(rel, thr2, ap, aq)) {
                                A[p * ld + q] = make_float2(0.f, 0.f);
                                A[q * ld + p] = make_float2(0.f, 0.f);
                            } else {
                                rotation32(ap, aq, b, c, s);
                            }
                        }
                        const float4 ro = make_float4(c, s.x, s.y, __int_as_float(p | (q << 16)));
                        rr[i] = ro;
                        if (grec != nullptr) grec[(size_t)(total + r) * npair + i] = ro;
                    }
                    asm volatile("bar.sync 1, %0;" ::"r"(ja) : "memory");
                    // warp task j: block row a = j (blocks b = 0 .. a) followed by block row npair - 1 - j
                    // (blocks 0 .. npair - 1 - j): npair + 1 blocks, lanes over them
                    for (int j = warp; j < (npair + 1) / 2; j += ja / 32) {
                        for (int l = lane; l < npair + 1; l += 32) {
                            int a = j, b = l;
                            if (l > j) { a = npair - 1 - j; b = l - j - 1; }
                            if (a == j && l > j) continue;   // odd npair: the middle row is taken once
                            const float4 ra = rr[a], rb = rr[b];
                            if (ra.y == 0.f && ra.z == 0.f && rb.y == 0.f && rb.z == 0.f) continue;   // both identity
                            const int pqa = __float_as_int(ra.w), pqb = __float_as_int(rb.w);
                            const int pa = pqa & 0xffff, qa = pqa >> 16, pb = pqb & 0xffff, qb = pqb >> 16;
                            const bool va = qa < n, vb = qb < n;
                            float2* Ap = A + pa * ld;
                            float2* Aq = A + qa * ld;   // row qa = n (the dummy) is never accessed
                            const float2 z2 = make_float2(0.f, 0.f);
                            const float2 x00 = Ap[pb];
                            const float2 x01 = vb ? Ap[qb] : z2;
                            const float2 x10 = va ? Aq[pb] : z2;
                            const float2 x11 = va && vb ? Aq[qb] : z2;
                            const float ca = ra.x, cb = rb.x;
                            const float2 sa = make_float2(ra.y, ra.z), sb = make_float2(rb.y, rb.z);
                            const float2 sac = conjf2(sa), sbc = conjf2(sb);
                            // rows: J_a^H X;  columns: (J_a^H X) J_b
                            const float2 y00 = rot_l(ca, sa, x00, x10), y01 = rot_l(ca, sa, x01, x11);
                            const float2 y10 = rot_r(ca, sac, x00, x10), y11 = rot_r(ca, sac, x01, x11);
                            const float2 z00 = rot_l(cb, sbc, y00, y01), z01 = rot_r(cb, sb, y00, y01);
                            const float2 z10 = rot_l(cb, sbc, y10, y11), z11 = rot_r(cb, sb, y10, y11);
                            if (a != b) {   // the block and its mirror image
                                Ap[pb] = z00; A[pb * ld + pa] = conjf2(z00);
                                if (vb) { Ap[qb] = z01; A[qb * ld + pa] = conjf2(z01); }
                                if (va) { Aq[pb] = z10; A[pb * ld + qa] = conjf2(z10); }
                                if (va && vb) { Aq[qb] = z11; A[qb * ld + qa] = conjf2(z11); }
                            } else {
                                Ap[pa] = z00;
                                if (va) { Aq[pa] = z10; Ap[qa] = conjf2(z10); Aq[qa] = z11; }
                            }
                        }
                    }
                    asm volatile("bar.sync 1, %0;" ::"r"(ja) : "memory");
                }
                if (last) {   // the next sweep rotates only pairs above the threshold: stop when there are none
                    for (int e = tid; e < n * n; e += ja) {
                        const int r = e / n, cc = e % n;
                        if (r > cc) {
                            const float2 b = A[r * ld + cc];
                            above |= fmaf(b.x, b.x, b.y * b.y) > jac_lim(rel, thr2, A[r * ld + r].x, A[cc * ld + cc].x);
                        }
                    }
                }
            } else if (pend) {
                jacobi_apply_v(V, n, vrs, vcs, rec + (size_t)(buf ^ 1) * C * npair, pend, pend_r0);
            }
            const int any = __syncthreads_or(above);
            pend = nr; pend_r0 = r0; buf ^= 1;
            total += nr;
            if (last && !any) done = true;
        }
    }
    if (!agroup && pend) jacobi_apply_v(V, n, vrs, vcs, rec + (size_t)(buf ^ 1) * C * npair, pend, pend_r0);
    if (grec != nullptr && tid == 0) *nrec = total;
    __syncthreads();
    return sweep;
}

__device__ __forceinline__ void jacobi_load(const cplx* R, double scale, float2* A, float2* V, int n, int ld) {
    for (int e = threadIdx.x; e < n * n; e += JT) {
        const int r = e / n, cc = e % n;
        const double2 v = R[e];
        A[r * ld + cc] = make_float2((float)(v.x * scale), (float)(v.y * scale));
        if (V != nullptr) V[r * ld + cc] = make_float2(r == cc ? 1.f : 0.f, 0.f);
    }
}

__device__ __forceinline__ float jacobi_fro2(const float2* A, int n, int ld) {
    float f = 0.f;
    for (int e = threadIdx.x; e < n * n; e += JT) { const float2 a = A[(e / n) * ld + e % n]; f += a.x * a.x + a.y * a.y; }
    return f;
}

// W = V^H - dsub I: row j is the conjugate of eigenvector j (dsub = 1 stores the re-seed as a correction);
// element (k, j) of V at V[k * rs + j * cs]
__device__ __forceinline__ void jacobi_store(const float2* V, cplx* Ws, int n, int rs, int cs, double dsub) {
    for (int e = threadIdx.x; e < n * n; e += JT) {
        const int j = e / n, k = e % n;
        const float2 v = V[k * rs + j * cs];
        Ws[e] = make_double2((double)v.x - (k == j ? dsub : 0.0), -v.y);
    }
}

// FP32 Jacobi per sector.  Dynamic shared memory (`smem` bytes): A and V of sectors with n <= kSmemMaxN
// (A alone for n <= kSmemMaxA, V then in `gwork`, transposed), then the rotation record; larger sectors
// keep A and V in `gwork`.
//  - seed (rel = false): src = rho; writes W0 = X0^H (X0: unsorted eigenvector columns), ||rho||_F, the
//    initial iteration count, and clears the sector's re-seed flag;
//  - re-seed (rel = true) in refinement iteration `it`, for sectors whose flag is set: src = S = X^H rho X
//    scaled by 1 / ||rho||_F, so that eigenvalues far below FP32's resolution of rho are resolved relative
//    to their own size; writes V^H - I (V: eigenvectors of S) over the correction dst = E1h, so that the
//    iteration's update is W <- V^H W, and asks for two more refinements.
__global__ void __launch_bounds__(JT) k_jacobi32(const cplx* __restrict__ src, cplx* __restrict__ dst,
                                                 double* __restrict__ rho_fro, int* __restrict__ n_iter,
                                                 int* __restrict__ flags, EigTables tb, float2* __restrict__ gwork,
                                                 float4* __restrict__ grec, int* __restrict__ nrec,
                                                 int smem, bool rel, int it, int2* __restrict__ stats) {
    pdl_enter();
    const long long t_start = clock64();
    extern __shared__ float4 fsm4[];
    float2* fsm = reinterpret_cast<float2*>(fsm4);
    const int sct = blockIdx.x, n = tb.dims[sct], tid = threadIdx.x;
    const int mode = jac_mode(n);
    if (rel && (it >= *n_iter || flags[sct] == 0)) {   // iteration skipped, or nothing to re-seed
        if (jac_recorded(n) && tid == 0) nrec[sct] = -1;   // nor is there anything to replay
        return;
    }
    const int64_t off = tb.off[sct];
    const int ld = n | 1;   // odd row stride: column accesses of a warp hit distinct banks
    float2* gA = gwork + 4 * off;
    float2* gV = gA + (int64_t)n * ld;   // transposed: element (k, p) at gV[p * ld + k]
    (void)gV;
    float4* rec = fsm4 + jac_base_bytes(n) / 16;
    const int C = jac_chunk(n, smem);
    __shared__ float red[JT / 32];
    __shared__ float thr_s;
    const double scale = rel ? 1.0 / rho_fro[sct] : 1.0;
    if (!rel && sct == 0 && tid == 0) *n_iter = kRefine;
    float fro;
    // V starts as the identity (record modes form V afterwards, in k_jacobi_replay)
    if (mode == JAC_SMEM) { jacobi_load(src + off, scale, fsm, fsm + n * ld, n, ld); __syncthreads(); fro = jacobi_fro2(fsm, n, ld); }
    else if (mode == JAC_SMEM_A) { jacobi_load(src + off, scale, fsm, nullptr, n, ld); __syncthreads(); fro = jacobi_fro2(fsm, n, ld); }
    else { jacobi_load(src + off, scale, gA, nullptr, n, ld); __syncthreads(); fro = jacobi_fro2(gA, n, ld); }
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
    if ((tid & 31) == 0) red[tid >> 5] = fro;
    __syncthreads();
    if (tid == 0) {
        float f = 0.f;
        for (int k = 0; k < JT / 32; ++k) f += red[k];
        if (rel) {
            thr_s = kReseedFloor;          // S is in units of ||rho||_F
            flags[sct] = 0;
            atomicMax(n_iter, min(kOaIters, it + 3));
        } else {
            thr_s = 4.8e-7f * sqrtf(f);    // 4 eps_fp32 ||A||_F: above FP32 rounding noise, so sweeps terminate
            rho_fro[sct] = sqrtf(f);       // ||rho||_F for the refinement's cluster threshold
            flags[sct] = 0;
        }
    }
    __syncthreads();
    const float thr = thr_s;
    int sweeps;
    if (mode == JAC_SMEM) {
        sweeps = jacobi_sweeps(fsm, fsm + n * ld, n, ld, ld, 1, thr, rel, rec, C, JA, nullptr, nullptr);
        jacobi_store(fsm + n * ld, dst + off, n, ld, 1, rel ? 1.0 : 0.0);
    } else if (mode == JAC_SMEM_A) {   // dst is written by k_jacobi_replay
        sweeps = jacobi_sweeps(fsm, nullptr, n, ld, 1, ld, thr, rel, rec, C, JT, grec + tb.roff[sct], nrec + sct);
    } else {
        sweeps = jacobi_sweeps(gA, nullptr, n, ld, 1, ld, thr, rel, rec, C, JT, grec + tb.roff[sct], nrec + sct);
    }
    // per sector of the last launch: sweeps and SM cycles (a measurement aid; tdmrg_eig_stats)
    if (tid == 0 && !rel) stats[sct] = make_int2(sweeps, (int)min(clock64() - t_start, (long long)INT_MAX));
}

// V of the sectors beyond kSmemMaxN from their rotation record: V starts as the identity and every
// recorded rotation J_r acts on columns (p, q) of every row, so rows are independent: CTA (b, y) holds
// rows 8y .. 8y + 7 of V of big sector b in shared memory and replays all rounds on them, the record
// staged through shared memory a batch of rounds at a time.  Writes W = V^H - dsub I like jacobi_store
// (dsub = 1 for a re-seed).  Runs after each k_jacobi32 launch; nrec < 0 marks a skipped sector.
__global__ void __launch_bounds__(kReplayThreads) k_jacobi_replay(const float4* __restrict__ grec, const int* __restrict__ nrec,
                                                                  cplx* __restrict__ dst, EigTables tb, int batch, bool rel) {
    pdl_enter();
    const int sct = tb.big[blockIdx.x], n = tb.dims[sct];
    const int nr = nrec[sct];
    const int k0 = blockIdx.y * kReplayRows;
    if (nr < 0 || k0 >= n) return;
    const int rows = min(kReplayRows, n - k0), ld = n | 1;
    const int P = n + (n & 1), npair = P / 2;
    extern __shared__ float4 rsm4[];
    float4* rb = rsm4;                                        // batch rounds x npair records
    float2* vs = reinterpret_cast<float2*>(rsm4 + (size_t)batch * npair);   // rows x ld
    const int tid = threadIdx.x;
    for (int e = tid; e < rows * n; e += blockDim.x) vs[(e / n) * ld + e % n] = make_float2(k0 + e / n == e % n ? 1.f : 0.f, 0.f);
    const float4* rec = grec + tb.roff[sct];
    for (int b0 = 0; b0 < nr; b0 += batch) {
        const int nb = min(batch, nr - b0);
        __syncthreads();
        for (int e = tid; e < nb * npair; e += blockDim.x) rb[e] = rec[(size_t)b0 * npair + e];
        __syncthreads();
        for (int r = 0; r < nb; ++r) {
            // lanes over rows within a pair: the rows' accesses to one column hit distinct banks (odd ld)
            for (int x = tid; x < npair * rows; x += blockDim.x) {
                const int i = x / rows, k = x % rows;
                const float4 ro = rb[r * npair + i];
                if (ro.y == 0.f && ro.z == 0.f) continue;   // identity
                const int p = __float_as_int(ro.w) & 0xffff, q = __float_as_int(ro.w) >> 16;
                const float2 s = make_float2(ro.y, ro.z), sc = conjf2(s);
                float2* row = vs + k * ld;
                const float2 vp = row[p], vq = row[q];
                row[p] = rot_l(ro.x, sc, vp, vq);
                row[q] = rot_r(ro.x, s, vp, vq);
            }
            __syncthreads();
        }
    }
    __syncthreads();
    const double dsub = rel ? 1.0 : 0.0;
    cplx* W = dst + tb.off[sct];
    for (int e = tid; e < rows * n; e += blockDim.x) {   // W[j][k0 + k] = conj(V[k0 + k][j]) - dsub delta
        const int k = e % rows, j = e / rows;
        const float2 v = vs[k * ld + j];
        W[(int64_t)j * n + k0 + k] = make_double2((double)v.x - (j == k0 + k ? dsub : 0.0), -v.y);
    }
}

// Refinement on W = X^H, which turns every product into a plain or conjugate-transposed operand of the
// grouped GEMM: rho X = rho W^H, G = W W^H, S = W (rho X), and X <- X (I + E) is W <- (I + E)^H W, the
// last one in the GEMM's correction mode (E^H W in FP32, W added in FP64).
// The element-wise steps run on (sector, row chunk) CTAs: FP64 arithmetic is slow per SM, so one CTA
// per sector would leave the largest sector's elements on one SM.
constexpr int kRowChunks = 8;

__device__ __forceinline__ void chunk_rows(int n, int ch, int& r0, int& r1) {
    const int rows = (n + kRowChunks - 1) / kRowChunks;
    r0 = min(n, ch * rows);
    r1 = min(n, r0 + rows);
}

// Work items of the element-wise refinement kernels: kOaElems consecutive elements of one sector's
// n x n block (row-major), the items of a sector contiguous; one CTA of kOaThreads threads per item, each
// thread with kOaElems / kOaThreads elements whose loads are issued together.  Small CTAs with equal
// work: FP64 instructions of empty warps would still occupy the slow FP64 pipe.
constexpr int kOaThreads = 64;
constexpr int kOaElems = 256;
constexpr int kOaPer = kOaElems / kOaThreads;
struct OaTables {
    const int4* items;   // (sector, e0, e1, -)
    const int* first;    // per sector: its first item; first[ns] = number of items
    double* part;        // per item: partial squared norms (||S - diag(lambda)||^2, ||I - G||^2)
    double* delta;       // per sector: the cluster threshold of this iteration
    int* count;          // per sector: items done (reset by the last one)
};

// lambda_i = Re S_ii / Re G_ii for the item's diagonal elements and the item's partial squared Frobenius
// norms of S - diag(lambda) and R = I - G; the last item of a sector to finish sums the sector's
// partials in item order and writes delta = 2 (||S - diag(lambda)||_F + ||rho||_F ||R||_F).
__global__ void __launch_bounds__(kOaThreads) k_oa_norms(const cplx* __restrict__ S, const cplx* __restrict__ G,
                                                         double* __restrict__ lam, const double* __restrict__ rho_fro,
                                                         OaTables oa, const int* __restrict__ n_iter, int it, EigTables tb) {
    pdl_enter();
    if (it >= *n_iter) return;   // refinement already converged
    const int4 item = oa.items[blockIdx.x];
    const int sct = item.x, n = tb.dims[sct];
    const int64_t off = tb.off[sct], eo = tb.eoff[sct];
    __shared__ double red[2][kOaThreads / 32];
    double2 sv[kOaPer], g[kOaPer];
#pragma unroll
    for (int u = 0; u < kOaPer; ++u) {
        const int e = item.y + threadIdx.x + kOaThreads * u;
        if (e < item.z) { sv[u] = S[off + e]; g[u] = G[off + e]; }
    }
    double offS = 0.0, rr = 0.0;
#pragma unroll
    for (int u = 0; u < kOaPer; ++u) {
        const int e = item.y + threadIdx.x + kOaThreads * u;
        if (e < item.z) {
            const int i = e / n, j = e - i * n;
            if (i == j) {
                const double l = sv[u].x / g[u].x;
                lam[eo + i] = l;
                sv[u].x -= l;
            }
            offS += sv[u].x * sv[u].x + sv[u].y * sv[u].y;
            const double rx = (i == j ? 1.0 : 0.0) - g[u].x, ry = -g[u].y;
            rr += rx * rx + ry * ry;
        }
    }
    const int w = threadIdx.x >> 5;
    if (item.y + w * 32 < item.z) {   // warps without elements skip the FP64 shuffle tree
        for (int o = 16; o > 0; o >>= 1) {
            offS += __shfl_xor_sync(0xffffffffu, offS, o);
            rr += __shfl_xor_sync(0xffffffffu, rr, o);
        }
    }
    if ((threadIdx.x & 31) == 0) { red[0][w] = offS; red[1][w] = rr; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = red[0][0], b = red[1][0];
        for (int k = 1; k < kOaThreads / 32; ++k) { a += red[0][k]; b += red[1][k]; }
        oa.part[2 * blockIdx.x] = a;
        oa.part[2 * blockIdx.x + 1] = b;
        __threadfence();
        const int i0 = oa.first[sct], i1 = oa.first[sct + 1];
        if (atomicAdd(oa.count + sct, 1) == i1 - i0 - 1) {
            __threadfence();
            a = 0.0; b = 0.0;
            for (int k = i0; k < i1; ++k) { a += __ldcg(oa.part + 2 * k); b += __ldcg(oa.part + 2 * k + 1); }
            oa.delta[sct] = 2.0 * (sqrt(a) + rho_fro[sct] * sqrt(b));
            oa.count[sct] = 0;   // every item of the sector has arrived: ready for the next iteration
        }
    }
}

// The item's elements of E^H (the update adds the identity).  With S and R = I - G Hermitian and lambda real,
// the conjugate of E_ji = (S_ji + lambda_i R_ji) / (lambda_i - lambda_j) is
// (S_ij + lambda_i R_ij) / (lambda_i - lambda_j), and that of the cluster value R_ji / 2 is R_ij / 2.
__global__ void __launch_bounds__(kOaThreads) k_oa_update(const cplx* __restrict__ S, const cplx* __restrict__ G,
                                                          const double* __restrict__ lam, OaTables oa,
                                                          const double* __restrict__ rho_fro, cplx* __restrict__ E1h,
                                                          int* __restrict__ n_iter, int* __restrict__ flags, int it, EigTables tb) {
    pdl_enter();
    if (it >= *n_iter) return;   // refinement already converged
    const int4 item = oa.items[blockIdx.x];
    const int sct = item.x, n = tb.dims[sct];
    const int64_t off = tb.off[sct], eo = tb.eoff[sct];
    const double delta = oa.delta[sct], floor_s = (double)kReseedFloor * rho_fro[sct];
    double2 sv[kOaPer], g[kOaPer];
#pragma unroll
    for (int u = 0; u < kOaPer; ++u) {
        const int e = item.y + threadIdx.x + kOaThreads * u;
        if (e < item.z) { sv[u] = S[off + e]; g[u] = G[off + e]; }
    }
    bool big = false, clus = false;
    const bool orth_only = it >= kOaIters;   // E = R / 2: W <- (I + R / 2) W, a Newton-Schulz step
#pragma unroll
    for (int u = 0; u < kOaPer; ++u) {
        const int e = item.y + threadIdx.x + kOaThreads * u;
        if (e < item.z) {
            const int i = e / n, j = e - i * n;
            const double2 r = make_double2((i == j ? 1.0 : 0.0) - g[u].x, -g[u].y);
            double2 ev;
            const double li = lam[eo + i], lj = lam[eo + j];
            if (!orth_only && i != j && fabs(li - lj) > delta) {
                const double inv = 1.0 / (li - lj);
                ev = make_double2((sv[u].x + li * r.x) * inv, (sv[u].y + li * r.y) * inv);
            } else {
                ev = make_double2(0.5 * r.x, 0.5 * r.y);
                // clustered pair still coupled: the cluster is not diagonalised by this update
                if (i != j && !orth_only) clus |= fmax(fabs(sv[u].x), fabs(sv[u].y)) > floor_s;
            }
            big |= fmax(fabs(ev.x), fabs(ev.y)) > kTolE;
            E1h[off + e] = ev;   // the update adds the identity: W' = (I + E1h) W
        }
    }
    // from the last iteration that always runs on, a correction still above kTolE asks for one more; after
    // the last such iteration it asks for both orthonormalisation steps (an orthogonality error eps of W
    // becomes ~eps^2, then rounding), so that the eigenvectors always span an orthonormal basis
    if (it >= kRefine - 1 && it < kOaIters && __syncthreads_or(big) && threadIdx.x == 0)
        atomicMax(n_iter, it + 1 < kOaIters ? it + 2 : kMaxRefine);
    // at a re-seed iteration, a cluster with coupling above the floor sends the sector to the re-seed
    if (reseed_iter(it) && __syncthreads_or(clus) && threadIdx.x == 0) flags[sct] = 1;
}

// Order key of a double: unsigned comparison of keys is numeric comparison (-0 taken as +0).
__device__ __forceinline__ unsigned long long order_key(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v == 0.0 ? 0.0 : v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// Descending eigenvalue order (ties by index); rows of the chunk of U = X sorted, X = W^H (W after an even
// number of refinements is in W_even).
__global__ void __launch_bounds__(256) k_eig_sort(const cplx* __restrict__ W_even, const cplx* __restrict__ W_odd,
                                                  const int* __restrict__ n_iter, const double* __restrict__ lam,
                                                  cplx* __restrict__ U, double* __restrict__ evals, EigTables tb) {
    pdl_enter();
    const cplx* __restrict__ W = (*n_iter & 1) ? W_odd : W_even;   // the iterate after the last refinement
    const int sct = blockIdx.x, ch = blockIdx.y, n = tb.dims[sct];
    const int64_t off = tb.off[sct], eo = tb.eoff[sct];
    __shared__ unsigned long long key[kMaxEigN];
    __shared__ int src[kMaxEigN];
    int r0, r1;
    chunk_rows(n, ch, r0, r1);
    if (r0 >= r1) return;
    for (int j = threadIdx.x; j < n; j += blockDim.x) key[j] = order_key(lam[eo + j]);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const unsigned long long kj = key[j];
        int rank = 0;
        for (int m = 0; m < n; ++m) rank += (key[m] > kj) || (key[m] == kj && m < j);
        src[rank] = j;
        if (ch == 0) evals[eo + rank] = lam[eo + j];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < (r1 - r0) * n; e += blockDim.x) {
        const int r = r0 + e / n, k = e % n;
        const double2 v = W[off + (int64_t)src[k] * n + r];
        U[off + (int64_t)r * n + k] = make_double2(v.x, -v.y);
    }
}

}  // namespace

// Layout of a group's work-item buffer: items, first (padded to 16 B), per-item partials, per-sector delta
// and per-sector counters.
OaTables oa_tables(const EigGroup& g) {
    unsigned char* b = static_cast<unsigned char*>(g.oa);
    const size_t b_items = (size_t)g.noa * sizeof(int4), b_first = ((size_t)(g.ns + 1) * sizeof(int) + 15) & ~(size_t)15;
    double* part = reinterpret_cast<double*>(b + b_items + b_first);
    double* delta = part + 2 * (size_t)g.noa;
    return OaTables{reinterpret_cast<const int4*>(b), reinterpret_cast<const int*>(b + b_items), part, delta,
                    reinterpret_cast<int*>(delta + g.ns)};
}
size_t oa_bytes(int noa, int ns) {
    return (size_t)noa * sizeof(int4) + (((size_t)(ns + 1) * sizeof(int) + 15) & ~(size_t)15) +
           2 * (size_t)noa * sizeof(double) + (size_t)ns * sizeof(double) + (size_t)ns * sizeof(int);
}

// Buffer ids of the refinement GEMMs (all packed like rho).
enum { EB_RHO = BUF_EXTRA0, EB_W, EB_AX, EB_S, EB_G, EB_E, EB_WN };

// Cost model of the split into two groups, in SM cycles: the Jacobi seed of one sector (about 7 sweeps of
// n - 1 rounds; a round costs ~1300 + 12 n cycles with A and V in shared memory, ~40 n beyond) and the
// refinement of a sector spread over the GPU (3 iterations of 2 m^3 complex FP64 MACs at ~140 FMA per
// cycle chip-wide, m = n rounded up to the 16 x 16 x 16 tiles of the grouped GEMM).  Fitted to graph-replay
// timings of the split sizes on the L=32 m=400 and L=48 m=1000 blocks; it only decides the scheduling.
double jacobi_cost(int n) { return 7.0 * std::max(n - 1, 0) * (n <= kSmemMaxN ? 1300.0 + 12.0 * n : 40.0 * n); }
double refine_cost(int n) {
    const double m = 16.0 * ((n + 15) / 16);
    return 0.35 * m * m * m;
}

// Sectors of the first group (run on the second stream): the k with the longest Jacobi seeds, k chosen to
// minimise max(J_1 + R(first k), J_{k+1} + R(rest)) (J_i the i-th longest seed); empty when one group is
// predicted within 10 % of the best split.
std::vector<int> long_sectors(const std::vector<int>& dim) {
    const int ns = (int)dim.size();
    std::vector<int> order(ns);
    for (int k = 0; k < ns; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dim[a] > dim[b]; });
    double rall = 0.0;
    for (int k = 0; k < ns; ++k) rall += refine_cost(dim[k]);
    if (ns < 2) return {};
    const double one = jacobi_cost(dim[order[0]]) + rall;
    double best = one, rl = 0.0;
    int bestk = 0;
    for (int k = 1; k < ns; ++k) {
        rl += refine_cost(dim[order[k - 1]]);
        const double t = std::max(jacobi_cost(dim[order[0]]) + rl, jacobi_cost(dim[order[k]]) + rall - rl);
        if (t < best) { best = t; bestk = k; }
    }
    if (bestk == 0 || best > 0.9 * one) return {};
    std::vector<int> sel(order.begin(), order.begin() + bestk);
    std::sort(sel.begin(), sel.end());
    return sel;
}

int setup_group(tdmrg_ctx* c, const Side& L, const std::vector<int64_t>& goff, const std::vector<int64_t>& geoff,
                EigGroup& G) {
    const int ns = (int)G.sel.size();
    G.ns = ns;
    std::vector<int64_t> off(ns), eoff(ns), roff(ns, 0);
    std::vector<int> dim(ns), big;
    int64_t nrec_total = 0;
    int maxn_big = 0;
    for (int k = 0; k < ns; ++k) {
        const int q = G.sel[k], n = L.dim[q], P = n + (n & 1);
        off[k] = goff[q]; eoff[k] = geoff[q]; dim[k] = n;
        if (!jac_recorded(n)) continue;   // beyond kSmemMaxN: records of up to kMaxSweeps sweeps, V replayed
        roff[k] = nrec_total;
        nrec_total += (int64_t)kMaxSweeps * (P - 1) * (P / 2);
        big.push_back(k);
        maxn_big = std::max(maxn_big, n);
    }
    G.nbig = (int)big.size();
    G.maxn_big = maxn_big;
    G.grec_entries = nrec_total;
    G.tables_bytes = (size_t)ns * (3 * sizeof(int64_t) + sizeof(int)) + big.size() * sizeof(int);
    int rc = dev_alloc(c, (void**)&G.tables, G.tables_bytes, "eig tables");
    if (!rc) rc = dev_alloc(c, (void**)&G.fro, ((size_t)ns + 1) * sizeof(double), "eig workspace");
    if (!rc && nrec_total) rc = dev_alloc(c, (void**)&G.grec, (size_t)nrec_total * sizeof(float4), "eig rotation record");
    if (!rc) rc = dev_alloc(c, (void**)&G.nrec, (size_t)ns * sizeof(int), "eig rotation record");
    if (!rc) rc = dev_alloc(c, (void**)&G.stats, (size_t)ns * sizeof(int2), "eig statistics");
    if (!rc) rc = dev_alloc(c, (void**)&G.flags, (size_t)ns * sizeof(int), "eig workspace");
    if (rc) return rc;
    std::vector<unsigned char> host(G.tables_bytes);
    unsigned char* h = host.data();
    memcpy(h, off.data(), ns * sizeof(int64_t));
    memcpy(h + ns * sizeof(int64_t), eoff.data(), ns * sizeof(int64_t));
    memcpy(h + 2 * ns * sizeof(int64_t), roff.data(), ns * sizeof(int64_t));
    memcpy(h + 3 * ns * sizeof(int64_t), dim.data(), ns * sizeof(int));
    if (!big.empty()) memcpy(h + 3 * ns * sizeof(int64_t) + ns * sizeof(int), big.data(), big.size() * sizeof(int));
    rc = cuda_check(c, cudaMemcpy(G.tables, host.data(), host.size(), cudaMemcpyHostToDevice), "eig tables");
    if (rc) return rc;
    {   // work items of the element-wise refinement kernels (counters start at zero)
        std::vector<int4> items;
        std::vector<int> first(ns + 1);
        for (int k = 0; k < ns; ++k) {
            first[k] = (int)items.size();
            const int nn = dim[k] * dim[k];
            for (int e0 = 0; e0 < nn; e0 += kOaElems) items.push_back(make_int4(k, e0, std::min(nn, e0 + kOaElems), 0));
        }
        first[ns] = (int)items.size();
        G.noa = (int)items.size();
        const size_t bytes = oa_bytes(G.noa, ns);
        rc = dev_alloc(c, &G.oa, bytes, "eig work items");
        if (rc) return rc;
        std::vector<unsigned char> ho(bytes, 0);
        memcpy(ho.data(), items.data(), items.size() * sizeof(int4));
        memcpy(ho.data() + items.size() * sizeof(int4), first.data(), first.size() * sizeof(int));
        rc = cuda_check(c, cudaMemcpy(G.oa, ho.data(), bytes, cudaMemcpyHostToDevice), "eig work items");
        if (rc) return rc;
    }
    if (G.nbig) {   // replay: 8 rows of V and as many rounds of the record as fit in 48 KB of shared memory
        const int P = maxn_big + (maxn_big & 1);
        const int slab = kReplayRows * (maxn_big | 1) * (int)sizeof(float2);
        G.replay_batch = std::max(1, (48 * 1024 - slab) / ((P / 2) * (int)sizeof(float4)));
        G.replay_smem = G.replay_batch * (P / 2) * (int)sizeof(float4) + slab;
    }
    // task lists: AX = rho W^H; S = W AX and G = W W^H; W' = E1h W
    struct Prod { int cbuf, abuf, bbuf; int8_t opb, herm; };
    auto one = [&](TaskList& tl, std::initializer_list<Prod> prods) {
        tl.tasks.clear(); tl.segs.clear();
        for (int k = 0; k < ns; ++k) {
            const int n = dim[k];
            for (const Prod& pr : prods) {
                Task t{};
                t.c_off = off[k]; t.c_buf = (int8_t)pr.cbuf; t.ldc = n; t.M = n; t.N = n; t.beta = 0;
                t.herm = pr.herm;
                t.seg_begin = (int)tl.segs.size();
                // K in chunks of kKChunk: split-K over the chunks spreads a sector's FP64 work over
                // several SMs (the per-SM FP64 rate is the limit, not the tile count)
                for (int k0 = 0; k0 < n; k0 += kKChunk) {
                    Seg sg{};
                    sg.a_off = off[k] + k0; sg.a_buf = (int8_t)pr.abuf; sg.lda = n;
                    sg.b_off = off[k] + (pr.opb == OPB_N ? (int64_t)k0 * n : (int64_t)k0);
                    sg.b_buf = (int8_t)pr.bbuf; sg.ldb = n; sg.opb = pr.opb;
                    sg.K = std::min(kKChunk, n - k0); sg.scale = make_double2(1.0, 0.0); sg.dscale = -1;
                    tl.segs.push_back(sg);
                }
                t.seg_end = (int)tl.segs.size();
                tl.tasks.push_back(t);
            }
        }
        make_tiles(tl, kTileF64, kTileF64, kKChunk);
        return upload(c, tl);
    };
    // shared memory of the Jacobi launch: the most any sector asks for (A, V and a whole sweep of
    // rotation records), capped; every sector then holds at least one round of records
    int smem = 0;
    for (int k = 0; k < ns; ++k) {
        const int n = dim[k], P = n + (n & 1);
        smem = std::max(smem, jac_base_bytes(n) + 32 * (P / 2) * (P - 1));
    }
    G.jac_smem = std::min(smem, kJacSmemCap);
    for (int k = 0; k < ns && !rc; ++k)
        if (dim[k] > 1 && jac_chunk(dim[k], G.jac_smem) < 1) rc = fail(c, TDMRG_EINVAL, "rho_eig: Jacobi shared memory");
    // S = W rho W^H and G = W W^H are Hermitian: lower tiles plus mirror
    if (!rc) rc = one(G.tl_ax, {{EB_AX, EB_RHO, EB_W, OPB_C, 0}});
    if (!rc) rc = one(G.tl_sg, {{EB_S, EB_W, EB_AX, OPB_N, 1}, {EB_G, EB_W, EB_W, OPB_C, 1}});
    if (!rc) rc = one(G.tl_y, {{EB_WN, EB_E, EB_W, OPB_N, 0}});
    return rc;
}

// Seed, refinement and sort of one group's sectors on stream s.
cudaError_t launch_group(tdmrg_ctx* c, EigWork& w, EigGroup& G, const cplx* rho, double* evals, cplx* evecs, cudaStream_t s) {
    const int ns = G.ns;
    const int64_t* t64 = (const int64_t*)G.tables;
    const int* dims = (const int*)(t64 + 3 * ns);
    EigTables tb{t64, t64 + ns, t64 + 2 * ns, dims, dims + ns};
    // V of the record-mode sectors after each Jacobi launch (seed or re-seed)
    auto replay = [&](cplx* dst, bool rel) {
        if (!G.nbig) return;
        const dim3 grid(G.nbig, (G.maxn_big + kReplayRows - 1) / kReplayRows);
        launch_pdl(k_jacobi_replay, grid, kReplayThreads, G.replay_smem, s, G.grec, G.nrec, dst, tb, G.replay_batch, rel);
        c->launches++;
    };
    cplx* W = w.buf;
    cplx* Wn = w.buf + w.nrho;
    cplx* AX = w.buf + 2 * w.nrho;
    cplx* S = w.buf + 3 * w.nrho;
    cplx* Gm = w.buf + 4 * w.nrho;
    cplx* E1h = w.buf + 5 * w.nrho;
    int* n_iter = reinterpret_cast<int*>(G.fro + ns);
    const OaTables oat = oa_tables(G);
    launch_pdl(k_jacobi32, ns, JT, G.jac_smem, s, rho, W, G.fro, n_iter, G.flags, tb, w.gwork, G.grec, G.nrec, G.jac_smem,
               false, 0, G.stats);
    c->launches += 1;
    replay(W, false);
    GemmArgs a{};
    a.dscale = c->dscale;
    a.bufs[EB_RHO] = const_cast<cplx*>(rho);
    a.bufs[EB_AX] = AX; a.bufs[EB_S] = S; a.bufs[EB_G] = Gm; a.bufs[EB_E] = E1h;
    const cplx* W_even = W;
    const cplx* W_odd = Wn;
    int it = 0;
    // iterations past kRefine run on the device only when the previous correction asked for them
    auto gemm = [&](TaskList& tl, bool corr) {
        a.tasks = tl.d_tasks; a.segs = tl.d_segs; a.tiles = tl.d_tiles; a.ntiles = (int)tl.tiles.size();
        a.partials = tl.d_partials; a.counters = tl.d_counters;
        c->launches++;
        return launch_gemm_f64(a, s, it < kRefine ? nullptr : n_iter, it, corr);
    };
    const dim3 chunks(ns, kRowChunks);
    cudaError_t e = cudaGetLastError();
    for (; it < kMaxRefine && e == cudaSuccess; ++it) {
        a.bufs[EB_W] = W; a.bufs[EB_WN] = Wn;
        // the orthonormalisation steps need G = W W^H only (S is formed but not read, lambda stays)
        const bool orth_only = it >= kOaIters;
        if (!orth_only) e = gemm(G.tl_ax, false);
        if (e == cudaSuccess) e = gemm(G.tl_sg, false);
        if (G.noa) {
            if (!orth_only)
                launch_pdl(k_oa_norms, G.noa, kOaThreads, 0, s, S, Gm, w.lam, (const double*)G.fro, oat, n_iter, it, tb);
            launch_pdl(k_oa_update, G.noa, kOaThreads, 0, s, S, Gm, w.lam, oat, (const double*)G.fro, E1h, n_iter, G.flags,
                       it, tb);
        }
        if (reseed_iter(it)) {
            launch_pdl(k_jacobi32, ns, JT, G.jac_smem, s, S, E1h, G.fro, n_iter, G.flags, tb, w.gwork, G.grec, G.nrec,
                       G.jac_smem, true, it, G.stats);
            c->launches++;
            replay(E1h, true);
        }
        if (e == cudaSuccess) e = gemm(G.tl_y, true);
        if (G.noa) c->launches += orth_only ? 1 : 2;
        std::swap(W, Wn);
    }
    if (e == cudaSuccess) {
        launch_pdl(k_eig_sort, chunks, 256, 0, s, W_even, W_odd, n_iter, w.lam, evecs, evals, tb);
        c->launches++;
        e = cudaGetLastError();
    }
    return e;
}

int eig_prepare(tdmrg_ctx* c, int side) {
    const Side& L = c->side[side];
    const int ns = (int)L.dim.size();
    EigWork& w = c->eig[side];
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
        if (maxn > kMaxEigN) return fail(c, TDMRG_EINVAL, "rho_eig: sector dimension above 512");
        w.nrho = r; w.nev = e; w.maxn = maxn; w.ns = ns;
        int rc = dev_alloc(c, (void**)&w.buf, (size_t)6 * r * sizeof(cplx), "eig workspace");
        if (!rc) rc = dev_alloc(c, (void**)&w.lam, (size_t)e * sizeof(double), "eig workspace");
        if (!rc && maxn > kSmemMaxA) rc = dev_alloc(c, (void**)&w.gwork, (size_t)4 * r * sizeof(float2), "eig workspace");
        // the opt-in is a property of the kernel on the device, shared by every context: always the maximum
        if (!rc) rc = cuda_check(c, cudaFuncSetAttribute(k_jacobi32, cudaFuncAttributeMaxDynamicSharedMemorySize, kJacSmemCap),
                                 "eig smem");
        if (rc) return rc;
        // the longest Jacobi seeds on a second stream, beside the other sectors' seeds and refinement
        const std::vector<int> lng = long_sectors(L.dim);
        std::vector<char> in_long(ns, 0);
        for (int q : lng) in_long[q] = 1;
        w.ngroups = lng.empty() ? 1 : 2;
        w.grp[0].sel.clear();
        w.grp[1].sel.clear();
        for (int k = 0; k < ns; ++k) w.grp[w.ngroups == 2 && !in_long[k] ? 1 : 0].sel.push_back(k);
        for (int g = 0; g < w.ngroups && !rc; ++g) rc = setup_group(c, L, off, eoff, w.grp[g]);
        if (!rc && w.ngroups == 2) {
            rc = cuda_check(c, cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking), "eig stream");
            if (!rc) rc = cuda_check(c, cudaEventCreateWithFlags(&w.fork, cudaEventDisableTiming), "eig stream");
            if (!rc) rc = cuda_check(c, cudaEventCreateWithFlags(&w.join, cudaEventDisableTiming), "eig stream");
        }
        if (rc) return rc;
        w.ready = true;
    }
    return TDMRG_OK;
}

// `forked`: the second stream already follows the caller's stream (density_matrix with grouped = true).
int eig_launch(tdmrg_ctx* c, int side, const cplx* rho, double* evals, cplx* evecs, bool forked) {
    EigWork& w = c->eig[side];
    cudaStream_t s = c->stream;
    cudaError_t e = cudaSuccess;
    if (w.ngroups == 1) {
        e = launch_group(c, w, w.grp[0], rho, evals, evecs, s);
    } else {   // fork and join by events (kept as dependencies when the caller's stream is being captured)
        if (!forked) {
            e = cudaEventRecord(w.fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(w.side, w.fork, 0);
        }
        if (e == cudaSuccess) e = launch_group(c, w, w.grp[0], rho, evals, evecs, w.side);
        if (e == cudaSuccess) e = launch_group(c, w, w.grp[1], rho, evals, evecs, s);
        if (e == cudaSuccess) e = cudaEventRecord(w.join, w.side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, w.join, 0);
    }
    return cuda_check(c, e, "rho_eig launch");
}

int rho_eig(tdmrg_ctx* c, int side, const cplx* rho, double* evals, cplx* evecs) {
    const int rc = eig_prepare(c, side);
    return rc ? rc : eig_launch(c, side, rho, evals, evecs, false);
}

void release_eig(tdmrg_ctx* c, int side) {
    EigWork& w = c->eig[side];
    for (int g = 0; g < 2; ++g) {
        EigGroup& G = w.grp[g];
        release(c, G.tl_ax); release(c, G.tl_sg); release(c, G.tl_y);
        dev_free(c, G.tables, G.tables_bytes);
        dev_free(c, G.grec, (size_t)G.grec_entries * sizeof(float4));
        dev_free(c, G.nrec, (size_t)G.ns * sizeof(int));
        dev_free(c, G.stats, (size_t)G.ns * sizeof(int2));
        dev_free(c, G.fro, ((size_t)G.ns + 1) * sizeof(double));
        dev_free(c, G.flags, (size_t)G.ns * sizeof(int));
        dev_free(c, G.oa, oa_bytes(G.noa, G.ns));
    }
    dev_free(c, w.buf, (size_t)6 * w.nrho * sizeof(cplx));
    dev_free(c, w.lam, (size_t)w.nev * sizeof(double));
    dev_free(c, w.gwork, (size_t)4 * w.nrho * sizeof(float2));
    if (w.side) {   // work queued on the second stream ends before it is destroyed
        cudaStreamSynchronize(w.side);
        cudaStreamDestroy(w.side);
    }
    if (w.fork) cudaEventDestroy(w.fork);
    if (w.join) cudaEventDestroy(w.join);
    w = EigWork();
}

}  // namespace tdmrg

using namespace tdmrg;

extern "C" int tdmrg_eig_stats(tdmrg_ctx* c, int side, int32_t* sweeps, int64_t* cycles) {
    if (!c) return fail(nullptr, TDMRG_EINVAL, "null context");
    if (side != 0 && side != 1) return fail(c, TDMRG_EINVAL, "eig_stats: side must be 0 or 1");
    const EigWork& w = c->eig[side];
    if (!w.ready) return fail(c, TDMRG_ESTATE, "eig_stats: no eigendecomposition on this side yet");
    DeviceGuard g(c->opts.device);
    int rc = TDMRG_OK;
    for (int gi = 0; gi < w.ngroups && !rc; ++gi) {
        const EigGroup& G = w.grp[gi];
        std::vector<int2> h(G.ns);
        rc = cuda_check(c, cudaMemcpyAsync(h.data(), G.stats, G.ns * sizeof(int2), cudaMemcpyDeviceToHost, c->stream), "eig_stats");
        if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "eig_stats");
        for (int k = 0; k < G.ns && !rc; ++k) {
            if (sweeps) sweeps[G.sel[k]] = h[k].x;
            if (cycles) cycles[G.sel[k]] = h[k].y;
        }
    }
    return rc;
}
