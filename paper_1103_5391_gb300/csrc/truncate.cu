// Truncation of a block to m states and renormalisation of its operators into the kept basis (Sec. I:
// the block keeps the m most probable states of its reduced density matrix and every operator is
// carried along, O -> U^dag O U), the first pieces of a sweep on the GPU.
//
// Kept set: the m largest eigenvalues of rho over all sectors; eigenvalues within 1e-12 lambda_max of
// the m-th largest are ties, broken by (sector index, eigen index) ascending, so every sector keeps a
// prefix of its descending eigenvalues.  One CTA: the m-th largest value is found by bisection over
// order-preserving 64-bit keys, counting with one binary search per sector (each sector's eigenvalues
// are sorted), so the number of eigenvalues is not limited by shared memory.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace tdmrg {
namespace {

constexpr int TT = 256;   // threads of the truncation CTA

// Unsigned comparison of keys is numeric comparison of the doubles (-0 taken as +0).
__device__ __forceinline__ unsigned long long okey(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v == 0.0 ? 0.0 : v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// entries of the descending list ev[0..n) with key >= k
__device__ __forceinline__ int count_ge(const double* ev, int n, unsigned long long k) {
    int lo = 0, hi = n;   // ev[lo..) unknown; the list is descending, so keys are non-increasing
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (okey(ev[mid]) >= k) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// entries of ev with value > x (descending list)
__device__ __forceinline__ int count_gt(const double* ev, int n, double x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ev[mid] > x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ long long block_sum_ll(long long v, long long* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    long long s = 0;
    for (int w = 0; w < TT / 32; ++w) s += sh[w];
    return s;
}

__global__ void __launch_bounds__(TT) k_truncate(const double* __restrict__ evals, const int64_t* __restrict__ eoff,
                                                 const int* __restrict__ dims, int ns, int m, double tie_rel,
                                                 int* __restrict__ kept, double* __restrict__ discarded) {
    pdl_enter();
    __shared__ long long sh[TT / 32];
    __shared__ double dsh[TT / 32];
    __shared__ double lam_max;
    const int tid = threadIdx.x;
    long long total = 0;
    double mx = -1.0e308;
    for (int s = tid; s < ns; s += TT) {
        total += dims[s];
        if (dims[s] > 0) mx = fmax(mx, evals[eoff[s]]);
    }
    total = block_sum_ll(total, sh);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((tid & 31) == 0) dsh[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
        double v = dsh[0];
        for (int w = 1; w < TT / 32; ++w) v = fmax(v, dsh[w]);
        lam_max = v;
    }
    __syncthreads();
    if (total <= m) {   // everything is kept
        for (int s = tid; s < ns; s += TT) kept[s] = dims[s];
        if (discarded != nullptr && tid == 0) *discarded = 0.0;
        return;
    }
    // largest key k with #{key(lambda) >= k} >= m: the key of the m-th largest eigenvalue
    unsigned long long lo = 0ull, hi = ~0ull;   // invariant: count(lo) >= m, count(hi + 1) < m
    for (int it = 0; it < 64 && lo < hi; ++it) {
        const unsigned long long mid = lo + ((hi - lo) >> 1) + 1;   // in (lo, hi]
        long long c = 0;
        for (int s = tid; s < ns; s += TT) c += count_ge(evals + eoff[s], dims[s], mid);
        c = block_sum_ll(c, sh);
        if (c >= m) lo = mid;
        else hi = mid - 1;
    }
    // lambda_m: the eigenvalue whose key is lo (any sector holding it)
    __shared__ double lam_m;
    if (tid == 0) lam_m = 0.0;
    __syncthreads();
    for (int s = tid; s < ns; s += TT) {
        const int c = count_ge(evals + eoff[s], dims[s], lo);
        if (c > 0 && okey(evals[eoff[s] + c - 1]) == lo) lam_m = evals[eoff[s] + c - 1];   // same value everywhere
    }
    __syncthreads();
    const double tol = tie_rel * fmax(lam_max, 0.0);
    const double up = lam_m + tol;
    // per sector: states strictly above the tie band, and the tied states after them
    __shared__ int s_above[1024], s_tied[1024];   // ns <= 1024 (checked by the entry point)
    long long above = 0;
    for (int s = tid; s < ns; s += TT) {
        const double* ev = evals + eoff[s];
        const int a = count_gt(ev, dims[s], up);
        int b = a;   // tied: |lambda - lambda_m| <= tol, contiguous after the `a` larger ones
        while (b < dims[s] && fabs(ev[b] - lam_m) <= tol) ++b;
        s_above[s] = a;
        s_tied[s] = b - a;
        above += a;
    }
    above = block_sum_ll(above, sh);
    if (tid == 0) {   // ties to the lowest sectors first (sector order, then eigen order inside a sector)
        long long need = m - above;
        for (int s = 0; s < ns; ++s) {
            const int take = (int)(need < (long long)s_tied[s] ? need : (long long)s_tied[s]);
            kept[s] = s_above[s] + take;
            need -= take;
        }
    }
    __syncthreads();
    if (discarded != nullptr) {   // dropped weight, summed per sector in order, then over sectors in order
        double w = 0.0;
        for (int s = tid; s < ns; s += TT) {
            const double* ev = evals + eoff[s];
            double ws = 0.0;
            for (int k = kept[s]; k < dims[s]; ++k) ws += ev[k];
            w += ws;   // thread tid sums sectors tid, tid + TT, ... in order
        }
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        __syncthreads();
        if ((tid & 31) == 0) dsh[tid >> 5] = w;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < TT / 32; ++q) t += dsh[q];
            *discarded = t;
        }
    }
}

}  // namespace
}  // namespace tdmrg

using namespace tdmrg;

extern "C" int tdmrg_truncate_side(tdmrg_ctx* c, int side, const double* evals, int m, int32_t* kept, double* discarded) {
    if (!c) return fail(nullptr, TDMRG_EINVAL, "null context");
    if ((side != 0 && side != 1) || !evals || !kept || m < 1)
        return fail(c, TDMRG_EINVAL, "truncate: side not 0 or 1, null pointer or m < 1");
    const Side& L = c->side[side];
    if (!L.set) return fail(c, TDMRG_ESTATE, "truncate: block not set");
    const int ns = (int)L.dim.size();
    if (ns > 1024) return fail(c, TDMRG_EINVAL, "truncate: more than 1024 sectors");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->opts.device) cudaSetDevice(c->opts.device);
    std::vector<int64_t> eoff(ns);
    int64_t e = 0;
    for (int s = 0; s < ns; ++s) { eoff[s] = e; e += L.dim[s]; }
    // sector tables on the device (a few KB; reallocated only when the left block changes size)
    const size_t bytes = (size_t)ns * (sizeof(int64_t) + sizeof(int));
    int rc = TDMRG_OK;
    if (c->trunc_tables_bytes < bytes) {
        dev_free(c, c->trunc_tables, c->trunc_tables_bytes);
        c->trunc_tables = nullptr;
        c->trunc_tables_bytes = 0;
        rc = dev_alloc(c, &c->trunc_tables, bytes, "truncation tables");
        if (!rc) c->trunc_tables_bytes = bytes;
    }
    std::vector<unsigned char> host(bytes);
    memcpy(host.data(), eoff.data(), ns * sizeof(int64_t));
    memcpy(host.data() + ns * sizeof(int64_t), L.dim.data(), ns * sizeof(int));
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(c->trunc_tables, host.data(), bytes, cudaMemcpyHostToDevice, c->stream),
                             "truncation tables");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "truncation tables");
    if (!rc) {
        const int64_t* d_eoff = (const int64_t*)c->trunc_tables;
        const int* d_dims = (const int*)(d_eoff + ns);
        launch_pdl(k_truncate, 1, TT, 0, c->stream, evals, d_eoff, d_dims, ns, m, 1e-12, (int*)kept, discarded);
        c->launches++;
        rc = cuda_check(c, cudaGetLastError(), "truncate launch");
    }
    if (prev >= 0 && prev != c->opts.device) cudaSetDevice(prev);
    return rc;
}

extern "C" int tdmrg_truncate(tdmrg_ctx* c, const double* evals, int m, int32_t* kept, double* discarded) {
    return tdmrg_truncate_side(c, 0, evals, m, kept, discarded);
}

extern "C" int tdmrg_renormalize_op(tdmrg_ctx* c, int side, int op_id, const tdmrg_c64* U, const int32_t* kept,
                                    tdmrg_c64* out, int* nblk_out) {
    if (!c) return fail(nullptr, TDMRG_EINVAL, "null context");
    if ((side != 0 && side != 1) || !U || !kept || !out) return fail(c, TDMRG_EINVAL, "renormalize_op: bad argument");
    const Side& S = c->side[side];
    if (!S.set) return fail(c, TDMRG_ESTATE, "renormalize_op: block not set");
    auto it = c->ops[side].find(op_id);
    if (it == c->ops[side].end()) return fail(c, TDMRG_EINVAL, "renormalize_op: op id not set");
    const int ns = (int)S.dim.size();
    for (int s = 0; s < ns; ++s)
        if (kept[s] < 0 || kept[s] > S.dim[s]) return fail(c, TDMRG_EINVAL, "renormalize_op: kept count outside 0..dim");
    std::vector<int64_t> uoff(ns);
    int64_t u = 0;
    for (int s = 0; s < ns; ++s) { uoff[s] = u; u += (int64_t)S.dim[s] * S.dim[s]; }
    // stage 1: T = O U_in[:, :k_in] (stored as T^T); stage 2: O'^T = T^T conj(U_out[:, :k_out]) stored
    // transposed, i.e. O' = U_out^dag O U_in row-major
    TaskList s1, s2;
    int64_t scr = 0, o = 0;
    int nblk = 0;
    for (const auto& blk : it->second.blocks) {
        const int qo = std::get<0>(blk), qi = std::get<1>(blk);
        const int64_t boff = std::get<2>(blk);
        const int dO = S.dim[qo], dI = S.dim[qi], kO = kept[qo], kI = kept[qi];
        if (kO == 0 || kI == 0) continue;
        Task t1{};
        t1.c_off = scr; t1.c_buf = BUF_SCRATCH; t1.ldc = dO; t1.M = dO; t1.N = kI; t1.trans = 1;
        t1.seg_begin = (int)s1.segs.size();
        Seg a{};
        a.a_off = boff; a.a_buf = BUF_OPS; a.lda = dI;
        a.b_off = uoff[qi]; a.b_buf = BUF_IN; a.ldb = dI; a.opb = OPB_N;
        a.K = dI; a.scale = make_double2(1.0, 0.0); a.dscale = -1;
        s1.segs.push_back(a);
        t1.seg_end = (int)s1.segs.size();
        s1.tasks.push_back(t1);
        Task t2{};
        t2.c_off = o; t2.c_buf = BUF_OUT; t2.ldc = kI; t2.M = kI; t2.N = kO; t2.trans = 1;
        t2.seg_begin = (int)s2.segs.size();
        Seg b{};
        b.a_off = scr; b.a_buf = BUF_SCRATCH; b.lda = dO;
        b.b_off = uoff[qo]; b.b_buf = BUF_IN; b.ldb = dO; b.opb = OPB_CN;
        b.K = dO; b.scale = make_double2(1.0, 0.0); b.dscale = -1;
        s2.segs.push_back(b);
        t2.seg_end = (int)s2.segs.size();
        s2.tasks.push_back(t2);
        scr += (int64_t)dO * kI;
        o += (int64_t)kO * kI;
        ++nblk;
    }
    if (nblk_out) *nblk_out = nblk;
    if (nblk == 0) return TDMRG_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->opts.device) cudaSetDevice(c->opts.device);
    make_tiles(s1, kTileF64, kTileF64, kSplitK);
    make_tiles(s2, kTileF64, kTileF64, kSplitK);
    cplx* T = nullptr;
    int rc = dev_alloc(c, (void**)&T, (size_t)scr * sizeof(cplx), "renormalisation scratch");
    if (!rc) rc = upload(c, s1);
    if (!rc) rc = upload(c, s2);
    if (!rc) {
        GemmArgs g{};
        g.bufs[BUF_OPS] = c->pool;
        g.bufs[BUF_IN] = (cplx*)U;
        g.bufs[BUF_SCRATCH] = T;
        g.bufs[BUF_OUT] = (cplx*)out;
        g.dscale = c->dscale;
        for (TaskList* tl : {&s1, &s2}) {
            g.tasks = tl->d_tasks; g.segs = tl->d_segs; g.tiles = tl->d_tiles; g.ntiles = (int)tl->tiles.size();
            g.partials = tl->d_partials; g.counters = tl->d_counters;
            c->launches++;
            rc = cuda_check(c, launch_gemm_f64(g, c->stream, nullptr, 0), "renormalisation launch");
            if (rc) break;
        }
    }
    // the task lists and the scratch are released once the products are done
    int rc2 = cuda_check(c, cudaStreamSynchronize(c->stream), "renormalisation");
    release(c, s1);
    release(c, s2);
    dev_free(c, T, (size_t)scr * sizeof(cplx));
    if (prev >= 0 && prev != c->opts.device) cudaSetDevice(prev);
    return rc ? rc : rc2;
}
