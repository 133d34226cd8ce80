// C ABI entry points of libtdmrg (declared and documented in include/tdmrg.h).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include <algorithm>

#include "internal.h"
#include "tdmrg_bench.h"

using namespace tdmrg;

namespace {
thread_local std::string g_err = "no error";
}

namespace tdmrg {

int fail(tdmrg_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    else g_err = msg;
    return code;
}

int cuda_check(tdmrg_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return TDMRG_OK;
    return fail(c, TDMRG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int dev_alloc(tdmrg_ctx* c, void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) return TDMRG_OK;
    if (c->opts.hbm_budget && c->allocated + bytes > c->opts.hbm_budget)
        return fail(c, TDMRG_ENOMEM, std::string(what) + ": HBM budget exceeded");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, TDMRG_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    c->allocated += bytes;
    c->alloc_calls++;
    c->alloc_bytes += (int64_t)bytes;
    return TDMRG_OK;
}

void dev_free(tdmrg_ctx* c, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    c->allocated -= std::min(bytes, c->allocated);
}

}  // namespace tdmrg

namespace {

void drop_plans(tdmrg_ctx* c) {
    for (auto& kv : c->plans) {
        release(c, kv.second->stage1);
        release(c, kv.second->stage2);
        release(c, kv.second->thin[0]);
        release(c, kv.second->thin[1]);
        release_oz(c, kv.second->oz);
    }
    c->plans.clear();
    for (auto& kv : c->rho_plans) release(c, *kv.second);
    c->rho_plans.clear();
    for (auto& kv : c->dsum_norms) dev_free(c, kv.second.d, kv.second.bytes);
    c->dsum_norms.clear();
    release_corr(c);
}

void drop_krylov(tdmrg_ctx* c) {
    for (auto& kv : c->krylov) {
        KrylovWork& k = kv.second;
        size_t n = (size_t)k.n;
        dev_free(c, k.V, (k.nk + 1) * n * sizeof(cplx));
        dev_free(c, k.w, n * sizeof(cplx));
        dev_free(c, k.partA, 64 * kRedBlocks * sizeof(double2));
        dev_free(c, k.partB, 64 * kRedBlocks * sizeof(double2));
        dev_free(c, k.tri, 128 * sizeof(double));
        dev_free(c, k.flags, 4 * sizeof(int));
        dev_free(c, k.coef, (16 + 32) * 32 * sizeof(cplx));
        dev_free(c, k.bar, 4 * sizeof(unsigned));
        dev_free(c, k.segmem, k.segmem_bytes);
    }
    c->krylov.clear();
    c->last_krylov = nullptr;
}

int check_ctx(tdmrg_ctx* c) { return c ? TDMRG_OK : fail(nullptr, TDMRG_EINVAL, "null context"); }

int check_op(tdmrg_ctx* c, int side, int id) {
    if (id < 0) return TDMRG_OK;
    if (!c->ops[side].count(id))
        return fail(c, TDMRG_EINVAL, std::string(side ? "right" : "left") + " op id " + std::to_string(id) + " is not set");
    return TDMRG_OK;
}

// Cached plan for (terms id, op ids, Q_in, Q_out); terms id 0 = Hamiltonian, 1 = single product.
int get_plan(tdmrg_ctx* c, int kind, int opL, int opR, int qa, int qb, int oa, int ob, Plan** out) {
    auto key = std::make_tuple(kind, opL, opR, qa, qb, oa, ob);
    auto it = c->plans.find(key);
    if (it != c->plans.end()) { *out = it->second.get(); return TDMRG_OK; }
    std::vector<Term> terms;
    if (kind == 0) terms = c->ham;
    else terms.push_back({opL, opR, make_double2(1.0, 0.0)});
    std::unique_ptr<Plan> p(new (std::nothrow) Plan());
    if (!p) return fail(c, TDMRG_ENOMEM, "host allocation");
    int rc = build_plan(c, terms, qa, qb, oa, ob, p.get());
    if (!rc && kind == 0 && c->opts.prec == TDMRG_OZAKI_BF16) rc = build_oz(c, p.get(), c->opts.ozaki_slices);
    if (rc) {
        release(c, p->stage1); release(c, p->stage2); release(c, p->thin[0]); release(c, p->thin[1]);
        release_oz(c, p->oz);
        return rc;
    }
    *out = p.get();
    c->plans[key] = std::move(p);
    return TDMRG_OK;
}

int ensure_tmp(tdmrg_ctx* c, int64_t n) {
    if (n <= c->tmp_cap) return TDMRG_OK;
    dev_free(c, c->tmp, c->tmp_cap * sizeof(cplx));
    c->tmp = nullptr; c->tmp_cap = 0;
    int rc = dev_alloc(c, (void**)&c->tmp, n * sizeof(cplx), "expectation workspace");
    if (!rc) c->tmp_cap = n;
    return rc;
}

}  // namespace

namespace tdmrg {

int get_ham_plan(tdmrg_ctx* c, int a, int b, Plan** out) { return get_plan(c, 0, -1, -1, a, b, a, b, out); }

int check_device_status(tdmrg_ctx* c) {
    int st = 0;
    int rc = cuda_check(c, cudaMemcpy(&st, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost), "device status");
    if (rc) return rc;
    if (st) {
        cudaMemset(c->dstatus, 0, sizeof(int));
        return fail(c, TDMRG_ETIMEOUT, "a bounded device wait ran out (tensor-core mbarrier, Lanczos grid barrier or "
                                       "the wait probe); results are invalid");
    }
    return TDMRG_OK;
}

}  // namespace tdmrg

extern "C" {

void tdmrg_default_opts(tdmrg_opts* o) {
    if (!o) return;
    o->device = 0;
    o->stream = nullptr;
    o->prec = TDMRG_FP64;
    o->ozaki_slices = 4;
    o->nk_max = 16;
    o->breakdown_tol = 1e-12;
    o->hbm_budget = 0;
}

int tdmrg_create(tdmrg_ctx** out, const tdmrg_opts* o) {
    if (!out || !o) return fail(nullptr, TDMRG_EINVAL, "null argument to tdmrg_create");
    *out = nullptr;
    if (o->nk_max < 1 || o->nk_max > 32) return fail(nullptr, TDMRG_EINVAL, "nk_max must be in 1..32");
    if (o->prec != TDMRG_FP64 && o->prec != TDMRG_OZAKI_BF16) return fail(nullptr, TDMRG_EINVAL, "unsupported precision");
    if (o->prec == TDMRG_OZAKI_BF16 && (o->ozaki_slices < 2 || o->ozaki_slices > 6))
        return fail(nullptr, TDMRG_EINVAL, "ozaki_slices must be in 2..6");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || o->device < 0 || o->device >= ndev) {
        cudaGetLastError();
        return fail(nullptr, TDMRG_ECUDA, "no CUDA device " + std::to_string(o->device));
    }
    tdmrg_ctx* c = new (std::nothrow) tdmrg_ctx();
    if (!c) return fail(nullptr, TDMRG_ENOMEM, "host allocation");
    c->opts = *o;
    c->stream = (cudaStream_t)o->stream;
    DeviceGuard g(o->device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, o->device);
    int rc = dev_alloc(c, (void**)&c->red, 2 * 64 * kRedBlocks * sizeof(double2), "reduction workspace");
    if (!rc) rc = dev_alloc(c, (void**)&c->dscale, 64 * sizeof(double), "scale workspace");
    if (!rc) rc = dev_alloc(c, (void**)&c->dstatus, sizeof(int), "status word");
    if (!rc) rc = cuda_check(c, cudaMemset(c->dstatus, 0, sizeof(int)), "status word");
    if (rc) {
        g_err = c->err;
        tdmrg_destroy(c);
        return rc;
    }
    *out = c;
    return TDMRG_OK;
}

int tdmrg_destroy(tdmrg_ctx* c) {
    if (!c) return TDMRG_OK;
    DeviceGuard g(c->opts.device);
    cudaStreamSynchronize(c->stream);
    drop_plans(c);
    drop_krylov(c);
    release_eig(c, 0);
    release_eig(c, 1);
    dev_free(c, c->pool, c->pool_cap * sizeof(cplx));
    dev_free(c, c->scratch, c->scratch_cap * sizeof(cplx));
    dev_free(c, c->tmp, c->tmp_cap * sizeof(cplx));
    dev_free(c, c->red, 2 * 64 * kRedBlocks * sizeof(double2));
    dev_free(c, c->dsum_dscale, c->dsum_dscale_bytes);
    dev_free(c, c->dscale, 64 * sizeof(double));
    dev_free(c, c->dstatus, sizeof(int));
    dev_free(c, c->trunc_tables, c->trunc_tables_bytes);
    delete c;
    return TDMRG_OK;
}

int tdmrg_set_stream(tdmrg_ctx* c, void* stream) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    c->stream = (cudaStream_t)stream;
    c->opts.stream = stream;
    return TDMRG_OK;
}

int tdmrg_set_precision(tdmrg_ctx* c, int prec, int slices) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (prec != TDMRG_FP64 && prec != TDMRG_OZAKI_BF16) return fail(c, TDMRG_EINVAL, "unsupported precision " + std::to_string(prec));
    if (prec == TDMRG_OZAKI_BF16 && (slices < 2 || slices > 6)) return fail(c, TDMRG_EINVAL, "ozaki_slices must be in 2..6");
    DeviceGuard g(c->opts.device);
    cudaStreamSynchronize(c->stream);
    c->opts.prec = prec;
    c->opts.ozaki_slices = slices;
    drop_plans(c);   // plans are rebuilt in the new arithmetic
    return TDMRG_OK;
}

const char* tdmrg_last_error(tdmrg_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

int tdmrg_set_block(tdmrg_ctx* c, int side, int nsec, const int32_t* qn, const int32_t* dim) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if ((side != 0 && side != 1) || nsec < 1 || !qn || !dim) return fail(c, TDMRG_EINVAL, "set_block: bad argument");
    Side s;
    for (int k = 0; k < nsec; ++k) {
        if (dim[k] < 1) return fail(c, TDMRG_ESECTOR, "set_block: sector dimension < 1");
        if (k > 0) {
            bool asc = (qn[2 * k] > qn[2 * k - 2]) || (qn[2 * k] == qn[2 * k - 2] && qn[2 * k + 1] > qn[2 * k - 1]);
            if (!asc) return fail(c, TDMRG_ESECTOR, "set_block: sectors not strictly ascending");
        }
        s.nup.push_back(qn[2 * k]);
        s.ndn.push_back(qn[2 * k + 1]);
        s.dim.push_back(dim[k]);
        s.index[{qn[2 * k], qn[2 * k + 1]}] = k;
    }
    s.set = true;
    DeviceGuard g(c->opts.device);
    cudaStreamSynchronize(c->stream);
    release_eig(c, side);
    c->side[side] = s;
    c->ops[side].clear();
    c->dsum_src[0].clear();
    c->dsum_src[1].clear();
    c->dsum_nsrc = 0;
    c->ham_set = false;
    c->ham.clear();
    drop_plans(c);
    drop_krylov(c);
    if (!c->ops[0].size() && !c->ops[1].size()) c->pool_used = 0;
    return TDMRG_OK;
}

int tdmrg_set_op(tdmrg_ctx* c, int side, int id, int odd, int nblk, const int32_t* bq, const tdmrg_c64* data,
                 int on_device) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if ((side != 0 && side != 1) || id < 0 || nblk < 0 || (nblk > 0 && (!bq || !data)))
        return fail(c, TDMRG_EINVAL, "set_op: bad argument");
    const Side& S = c->side[side];
    if (!S.set) return fail(c, TDMRG_ESTATE, "set_op: block not set");
    BlockOp op;
    op.side = side;
    op.odd = odd ? 1 : 0;
    int64_t total = 0;
    std::vector<std::pair<int, int>> idx;
    for (int b = 0; b < nblk; ++b) {
        int qo = S.find(bq[4 * b], bq[4 * b + 1]), qi = S.find(bq[4 * b + 2], bq[4 * b + 3]);
        if (qo < 0 || qi < 0) return fail(c, TDMRG_ESECTOR, "set_op: block refers to an unknown sector");
        int dq = (bq[4 * b] + bq[4 * b + 1]) - (bq[4 * b + 2] + bq[4 * b + 3]);
        if (((dq & 1) != 0) != (op.odd != 0))
            return fail(c, TDMRG_ESECTOR, "set_op: block parity change does not match fermion_odd");
        for (auto& p : idx)
            if (p.first == qo && p.second == qi) return fail(c, TDMRG_ESECTOR, "set_op: duplicate block");
        idx.push_back({qo, qi});
        total += (int64_t)S.dim[qo] * S.dim[qi];
    }
    DeviceGuard g(c->opts.device);
    if (c->pool_used + total > c->pool_cap) {   // grow the pool (offsets stay valid)
        int64_t cap = std::max<int64_t>(2 * c->pool_cap, c->pool_used + total + 4096);
        cplx* np = nullptr;
        int rc = dev_alloc(c, (void**)&np, cap * sizeof(cplx), "operator pool");
        if (rc) return rc;
        if (c->pool_used) {
            rc = cuda_check(c, cudaMemcpyAsync(np, c->pool, c->pool_used * sizeof(cplx), cudaMemcpyDeviceToDevice,
                                               c->stream), "operator pool copy");
            if (rc) { dev_free(c, np, cap * sizeof(cplx)); return rc; }
        }
        cudaStreamSynchronize(c->stream);
        dev_free(c, c->pool, c->pool_cap * sizeof(cplx));
        c->pool = np;
        c->pool_cap = cap;
    }
    // real operator: every imaginary part is zero (checked on a host copy of device data)
    {
        std::vector<tdmrg_c64> hcopy;
        const tdmrg_c64* h = data;
        if (on_device && total) {
            hcopy.resize(total);
            // on the context's stream: device data the caller produced there is complete before it is read
            int rc = cuda_check(c, cudaMemcpyAsync(hcopy.data(), data, total * sizeof(tdmrg_c64), cudaMemcpyDeviceToHost,
                                                   c->stream), "set_op realness check");
            if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "set_op realness check");
            if (rc) return rc;
            h = hcopy.data();
        }
        op.real = 1;
        for (int64_t k = 0; k < total && op.real; ++k) op.real = h[k].im == 0.0;
    }
    int64_t off = c->pool_used;
    int64_t src = 0;
    for (int b = 0; b < nblk; ++b) {
        int64_t n = (int64_t)S.dim[idx[b].first] * S.dim[idx[b].second];
        op.blocks.push_back(std::make_tuple(idx[b].first, idx[b].second, off + src));
        src += n;
    }
    if (total) {
        int rc = cuda_check(c, cudaMemcpyAsync(c->pool + off, data, total * sizeof(cplx),
                                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
                            "set_op copy");
        if (rc) return rc;
        if (!on_device) cudaStreamSynchronize(c->stream);   // the caller may free its host buffer on return
    }
    c->pool_used += total;
    auto it = c->ops[side].find(id);
    op.version = it == c->ops[side].end() ? 0 : it->second.version + 1;
    c->ops[side][id] = op;
    drop_plans(c);
    return TDMRG_OK;
}

int tdmrg_set_hamiltonian(tdmrg_ctx* c, int hl, int hr, int nconn, const int32_t* opL, const int32_t* opR,
                          const tdmrg_c64* coeff) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!c->side[0].set || !c->side[1].set) return fail(c, TDMRG_ESTATE, "set_hamiltonian: blocks not set");
    if (nconn < 0 || (nconn > 0 && (!opL || !opR || !coeff))) return fail(c, TDMRG_EINVAL, "set_hamiltonian: bad argument");
    if (check_op(c, 0, hl) || check_op(c, 1, hr)) return TDMRG_EINVAL;
    std::vector<Term> terms;
    if (hl >= 0) {
        if (c->ops[0].at(hl).odd) return fail(c, TDMRG_EINVAL, "set_hamiltonian: H_L is fermion-odd");
        terms.push_back({hl, -1, make_double2(1.0, 0.0)});
    }
    if (hr >= 0) {
        if (c->ops[1].at(hr).odd) return fail(c, TDMRG_EINVAL, "set_hamiltonian: H_R is fermion-odd");
        terms.push_back({-1, hr, make_double2(1.0, 0.0)});
    }
    for (int k = 0; k < nconn; ++k) {
        if (opL[k] < 0 && opR[k] < 0) return fail(c, TDMRG_EINVAL, "set_hamiltonian: connection without operators");
        if (check_op(c, 0, opL[k]) || check_op(c, 1, opR[k])) return TDMRG_EINVAL;
        Term tm{opL[k], opR[k], make_double2(coeff[k].re, coeff[k].im)};
        tm.conn = k;
        terms.push_back(tm);
    }
    c->ham = terms;
    c->ham_set = true;
    c->dcoef = nullptr;   // a new Hamiltonian starts with its static coefficients
    c->ham_version++;
    drop_plans(c);
    return TDMRG_OK;
}

int tdmrg_sector_size(tdmrg_ctx* c, int a, int b, int64_t* out) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!out) return fail(c, TDMRG_EINVAL, "sector_size: null output");
    if (!c->side[0].set || !c->side[1].set) return fail(c, TDMRG_ESTATE, "sector_size: blocks not set");
    *out = sector_size(c, a, b);
    return TDMRG_OK;
}

int tdmrg_apply_h(tdmrg_ctx* c, int a, int b, const tdmrg_c64* psi, tdmrg_c64* out) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!c->ham_set) return fail(c, TDMRG_ESTATE, "apply_h: Hamiltonian not set");
    if (!psi || !out) return fail(c, TDMRG_EINVAL, "apply_h: null vector");
    DeviceGuard g(c->opts.device);
    Plan* p = nullptr;
    int rc = get_plan(c, 0, -1, -1, a, b, a, b, &p);
    if (rc) return rc;
    if (p->n_in == 0) return TDMRG_OK;
    return run_plan(c, *p, (const cplx*)psi, (cplx*)out, nullptr, 0);
}

int tdmrg_apply_op(tdmrg_ctx* c, int opL, int opR, int a, int b, const tdmrg_c64* psi, int oa, int ob,
                   tdmrg_c64* out) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!c->side[0].set || !c->side[1].set) return fail(c, TDMRG_ESTATE, "apply_op: blocks not set");
    if (!psi || !out) return fail(c, TDMRG_EINVAL, "apply_op: null vector");
    if (opL < 0 && opR < 0) return fail(c, TDMRG_EINVAL, "apply_op: both operators are the identity");
    if (check_op(c, 0, opL) || check_op(c, 1, opR)) return TDMRG_EINVAL;
    DeviceGuard g(c->opts.device);
    Plan* p = nullptr;
    int rc = get_plan(c, 1, opL, opR, a, b, oa, ob, &p);
    if (rc) return rc;
    if (p->n_out == 0) return TDMRG_OK;
    return run_plan(c, *p, (const cplx*)psi, (cplx*)out, nullptr, 0);
}

int tdmrg_evolve(tdmrg_ctx* c, int a, int b, const tdmrg_c64* phi, int n_v, const double* t_x, int nk,
                 tdmrg_c64* const* targets) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!c->ham_set) return fail(c, TDMRG_ESTATE, "evolve: Hamiltonian not set");
    if (!phi || !t_x || !targets || n_v < 1 || n_v > 16 || nk < 1 || nk > c->opts.nk_max)
        return fail(c, TDMRG_EINVAL, "evolve: bad argument (n_v in 1..16, nk in 1..nk_max)");
    for (int x = 0; x < n_v; ++x) {
        if (!targets[x]) return fail(c, TDMRG_EINVAL, "evolve: null target");
        if (!(t_x[x] >= 0.0) || !std::isfinite(t_x[x])) return fail(c, TDMRG_EINVAL, "evolve: t_x must be finite and >= 0");
        for (int y = 0; y < x; ++y)
            if (targets[x] == targets[y]) return fail(c, TDMRG_EINVAL, "evolve: targets alias each other");
    }
    DeviceGuard g(c->opts.device);
    return evolve(c, a, b, (const cplx*)phi, n_v, t_x, nk, (cplx* const*)targets);
}

int tdmrg_ground_state(tdmrg_ctx* c, int a, int b, tdmrg_c64* psi, int nk, int restarts, double* energy) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!c->ham_set) return fail(c, TDMRG_ESTATE, "ground_state: Hamiltonian not set");
    if (!psi || nk < 2 || nk > c->opts.nk_max || restarts < 1)
        return fail(c, TDMRG_EINVAL, "ground_state: bad argument (nk in 2..nk_max, restarts >= 1)");
    DeviceGuard g(c->opts.device);
    return ground_state(c, a, b, (cplx*)psi, nk, restarts, energy);
}

int tdmrg_evolve_segments(tdmrg_ctx* c, int a, int b, const tdmrg_c64* phi, int nseg, const int64_t* seg_len, int n_v,
                          const double* t_x, int nk, tdmrg_c64* const* targets) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!c->ham_set) return fail(c, TDMRG_ESTATE, "evolve_segments: Hamiltonian not set");
    if (!phi || !seg_len || !t_x || !targets || nseg < 1 || n_v < 1 || n_v > 16 || nk < 1 || nk > c->opts.nk_max)
        return fail(c, TDMRG_EINVAL, "evolve_segments: bad argument (n_v in 1..16, nk in 1..nk_max)");
    for (int x = 0; x < n_v; ++x)
        if (!targets[x] || !(t_x[x] >= 0.0)) return fail(c, TDMRG_EINVAL, "evolve_segments: null target or negative time");
    DeviceGuard g(c->opts.device);
    return evolve_segments(c, a, b, (const cplx*)phi, nseg, seg_len, n_v, t_x, nk, (cplx* const*)targets);
}

int tdmrg_evolve_segments_info(tdmrg_ctx* c, int a, int b, int nk, int nseg, int* nk_used, double* err) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    DeviceGuard g(c->opts.device);
    return segments_info(c, a, b, nk, nseg, nk_used, err);
}

// Direct sum of superblocks: the sectors of source k are moved apart (left n_up + 4096 k; right shifted so
// that source k's sector Q_k lands on Qsum = (4096 nsrc, 4096)), so that the products of the sum never
// pair blocks of different sources; operator ids become 2^20 k + id.
int tdmrg_direct_sum(tdmrg_ctx* dst, int nsrc, tdmrg_ctx* const* src, const int32_t* Q, int32_t* Qsum, int64_t* seg_off) {
    if (check_ctx(dst)) return TDMRG_EINVAL;
    if (nsrc < 1 || nsrc > 512 || !src || !Q) return fail(dst, TDMRG_EINVAL, "direct_sum: bad argument (1..512 sources)");
    constexpr int kShift = 4096, kIdStride = 1 << 20;
    for (int k = 0; k < nsrc; ++k) {
        const tdmrg_ctx* c = src[k];
        if (!c || c == dst) return fail(dst, TDMRG_EINVAL, "direct_sum: null source or the destination itself");
        if (!c->ham_set) return fail(dst, TDMRG_ESTATE, "direct_sum: a source has no Hamiltonian");
        if (c->dcoef) return fail(dst, TDMRG_EINVAL, "direct_sum: a source reads its coefficients at run time");
        if (c->opts.device != dst->opts.device) return fail(dst, TDMRG_EINVAL, "direct_sum: sources on another device");
        if (Q[2 * k] < 0 || Q[2 * k] >= kShift / 2 || Q[2 * k + 1] < 0 || Q[2 * k + 1] >= kShift / 2)
            return fail(dst, TDMRG_ESECTOR, "direct_sum: sector quantum numbers outside 0..2047");
        for (int sd = 0; sd < 2; ++sd)
            for (size_t q = 0; q < c->side[sd].dim.size(); ++q)
                if (c->side[sd].nup[q] < 0 || c->side[sd].nup[q] >= kShift / 2 || c->side[sd].ndn[q] < 0 ||
                    c->side[sd].ndn[q] >= kShift / 2)
                    return fail(dst, TDMRG_ESECTOR, "direct_sum: block quantum numbers outside 0..2047");
        for (const auto& kv : c->ops[0]) if (kv.first >= kIdStride) return fail(dst, TDMRG_EINVAL, "direct_sum: op id >= 2^20");
        for (const auto& kv : c->ops[1]) if (kv.first >= kIdStride) return fail(dst, TDMRG_EINVAL, "direct_sum: op id >= 2^20");
    }
    const int Bu = kShift * nsrc, Bd = kShift;
    auto shL = [&](int k) { return std::make_pair(kShift * k, 0); };
    auto shR = [&](int k) { return std::make_pair(Bu - Q[2 * k] - kShift * k, Bd - Q[2 * k + 1]); };
    // sector tables
    std::vector<int32_t> lq, ld;
    std::vector<std::pair<std::pair<int, int>, int>> rs;
    for (int k = 0; k < nsrc; ++k) {
        const Side& L = src[k]->side[0];
        const Side& R = src[k]->side[1];
        for (size_t q = 0; q < L.dim.size(); ++q) {
            lq.push_back(L.nup[q] + shL(k).first); lq.push_back(L.ndn[q] + shL(k).second); ld.push_back(L.dim[q]);
        }
        for (size_t q = 0; q < R.dim.size(); ++q) rs.push_back({{R.nup[q] + shR(k).first, R.ndn[q] + shR(k).second}, R.dim[q]});
    }
    std::sort(rs.begin(), rs.end());
    std::vector<int32_t> rq, rd;
    for (auto& e : rs) { rq.push_back(e.first.first); rq.push_back(e.first.second); rd.push_back(e.second); }
    int rc = tdmrg_set_block(dst, 0, (int)ld.size(), lq.data(), ld.data());
    if (!rc) rc = tdmrg_set_block(dst, 1, (int)rd.size(), rq.data(), rd.data());
    if (rc) return rc;
    DeviceGuard g(dst->opts.device);
    // operators: the blocks of every source operator, gathered from the source pool
    for (int k = 0; k < nsrc && !rc; ++k) {
        const tdmrg_ctx* c = src[k];
        cudaStreamSynchronize(c->stream);
        for (int sd = 0; sd < 2 && !rc; ++sd) {
            const Side& S = c->side[sd];
            const std::pair<int, int> sh = sd == 0 ? shL(k) : shR(k);
            for (const auto& kv : c->ops[sd]) {
                const BlockOp& op = kv.second;
                std::vector<int32_t> bq;
                int64_t tot = 0;
                for (const auto& blk : op.blocks) {
                    const int qo = std::get<0>(blk), qi = std::get<1>(blk);
                    bq.insert(bq.end(), {S.nup[qo] + sh.first, S.ndn[qo] + sh.second, S.nup[qi] + sh.first, S.ndn[qi] + sh.second});
                    tot += (int64_t)S.dim[qo] * S.dim[qi];
                }
                cplx* tmp = nullptr;
                rc = dev_alloc(dst, (void**)&tmp, (size_t)std::max<int64_t>(tot, 1) * sizeof(cplx), "direct sum gather");
                if (rc) break;
                int64_t o = 0;
                for (const auto& blk : op.blocks) {
                    const int64_t nb = (int64_t)S.dim[std::get<0>(blk)] * S.dim[std::get<1>(blk)];
                    if (!rc) rc = cuda_check(dst, cudaMemcpyAsync(tmp + o, c->pool + std::get<2>(blk), nb * sizeof(cplx),
                                                                  cudaMemcpyDeviceToDevice, dst->stream), "direct sum gather");
                    o += nb;
                }
                if (!rc) rc = tdmrg_set_op(dst, sd, kIdStride * k + kv.first, op.odd, (int)op.blocks.size(), bq.data(),
                                           (const tdmrg_c64*)tmp, 1);
                cudaStreamSynchronize(dst->stream);
                dev_free(dst, tmp, (size_t)std::max<int64_t>(tot, 1) * sizeof(cplx));
                if (rc) break;
            }
        }
    }
    if (rc) return rc;
    // Hamiltonian: every source's terms with its operator ids
    std::vector<Term> terms;
    for (int k = 0; k < nsrc; ++k)
        for (const Term& t : src[k]->ham) {
            Term u = t;
            u.opL = t.opL >= 0 ? kIdStride * k + t.opL : -1;
            u.opR = t.opR >= 0 ? kIdStride * k + t.opR : -1;
            u.conn = -1;
            terms.push_back(u);
        }
    dst->ham = terms;
    dst->ham_set = true;
    dst->dcoef = nullptr;
    dst->ham_version++;
    drop_plans(dst);
    // source of every sector (left sectors come in source order; right ones were sorted)
    dst->dsum_src[0].clear();
    for (int k = 0; k < nsrc; ++k) dst->dsum_src[0].insert(dst->dsum_src[0].end(), src[k]->side[0].dim.size(), k);
    dst->dsum_src[1].assign(dst->side[1].dim.size(), -1);
    for (int k = 0; k < nsrc; ++k) {
        const Side& R = src[k]->side[1];
        for (size_t q = 0; q < R.dim.size(); ++q)
            dst->dsum_src[1][dst->side[1].find(R.nup[q] + shR(k).first, R.ndn[q] + shR(k).second)] = k;
    }
    dst->dsum_nsrc = nsrc;
    if (Qsum) { Qsum[0] = Bu; Qsum[1] = Bd; }
    int64_t off = 0;
    for (int k = 0; k < nsrc; ++k) {
        if (seg_off) seg_off[k] = off;
        off += sector_size(src[k], Q[2 * k], Q[2 * k + 1]);
    }
    if (seg_off) seg_off[nsrc] = off;
    if (sector_size(dst, Bu, Bd) != off) return fail(dst, TDMRG_ESECTOR, "direct_sum: the summed sector does not add up");
    return TDMRG_OK;
}

int tdmrg_evolve_info(tdmrg_ctx* c, int* nk_used, double* err, double* alpha, double* beta) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!c->last_krylov) return fail(c, TDMRG_ESTATE, "evolve_info: no evolve yet");
    DeviceGuard g(c->opts.device);
    return evolve_info(c, nk_used, err, alpha, beta);
}

int tdmrg_tst_weights(int n_v, double* w_gs, double* w) {
    if (n_v < 2 || !w_gs || !w) return fail(nullptr, TDMRG_EINVAL, "tst_weights: n_v >= 2 and non-null outputs");
    const double omega = 1.0 / (double)(n_v + 1 + 3);
    *w_gs = 2.0 * omega;
    for (int x = 0; x < n_v; ++x) w[x] = omega;
    w[0] = 2.0 * omega;
    w[n_v - 1] = 2.0 * omega;
    return TDMRG_OK;
}

int tdmrg_rho_size_side(tdmrg_ctx* c, int side, int64_t* rho_entries, int64_t* n_evals) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (side != 0 && side != 1) return fail(c, TDMRG_EINVAL, "rho_size: side must be 0 or 1");
    if (!c->side[side].set) return fail(c, TDMRG_ESTATE, "rho_size: block not set");
    int64_t r = 0, e = 0;
    for (int d : c->side[side].dim) { r += (int64_t)d * d; e += d; }
    if (rho_entries) *rho_entries = r;
    if (n_evals) *n_evals = e;
    return TDMRG_OK;
}

int tdmrg_rho_size(tdmrg_ctx* c, int64_t* rho_entries, int64_t* n_evals) {
    return tdmrg_rho_size_side(c, 0, rho_entries, n_evals);
}

int tdmrg_density_matrix_side(tdmrg_ctx* c, int side, int nt, const int32_t* Q, const tdmrg_c64* const* psi,
                              const double* w, tdmrg_c64* rho) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!c->side[0].set || !c->side[1].set) return fail(c, TDMRG_ESTATE, "density_matrix: blocks not set");
    if ((side != 0 && side != 1) || nt < 1 || nt > kMaxBufs - BUF_EXTRA0 || !Q || !psi || !w || !rho)
        return fail(c, TDMRG_EINVAL, "density_matrix: bad argument (side 0 or 1, 1..12 targets)");
    for (int l = 0; l < nt; ++l)
        if (!psi[l] || !(w[l] >= 0.0)) return fail(c, TDMRG_EINVAL, "density_matrix: null state or negative weight");
    DeviceGuard g(c->opts.device);
    return density_matrix(c, side, nt, Q, (const cplx* const*)psi, w, (cplx*)rho);
}

int tdmrg_density_matrix(tdmrg_ctx* c, int nt, const int32_t* Q, const tdmrg_c64* const* psi, const double* w,
                         tdmrg_c64* rho) {
    return tdmrg_density_matrix_side(c, 0, nt, Q, psi, w, rho);
}

int tdmrg_rho_eig_side(tdmrg_ctx* c, int side, const tdmrg_c64* rho, double* evals, tdmrg_c64* evecs) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (side != 0 && side != 1) return fail(c, TDMRG_EINVAL, "rho_eig: side must be 0 or 1");
    if (!c->side[side].set) return fail(c, TDMRG_ESTATE, "rho_eig: block not set");
    if (!rho || !evals || !evecs) return fail(c, TDMRG_EINVAL, "rho_eig: null pointer");
    DeviceGuard g(c->opts.device);
    return rho_eig(c, side, (const cplx*)rho, evals, (cplx*)evecs);
}

int tdmrg_rho_eig(tdmrg_ctx* c, const tdmrg_c64* rho, double* evals, tdmrg_c64* evecs) {
    return tdmrg_rho_eig_side(c, 0, rho, evals, evecs);
}

int tdmrg_density_eig(tdmrg_ctx* c, int side, int nt, const int32_t* Q, const tdmrg_c64* const* psi, const double* w,
                      tdmrg_c64* rho, double* evals, tdmrg_c64* evecs) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!c->side[0].set || !c->side[1].set) return fail(c, TDMRG_ESTATE, "density_eig: blocks not set");
    if ((side != 0 && side != 1) || nt < 1 || nt > kMaxBufs - BUF_EXTRA0 || !Q || !psi || !w || !rho || !evals || !evecs)
        return fail(c, TDMRG_EINVAL, "density_eig: bad argument (side 0 or 1, 1..12 targets, non-null outputs)");
    for (int l = 0; l < nt; ++l)
        if (!psi[l] || !(w[l] >= 0.0)) return fail(c, TDMRG_EINVAL, "density_eig: null state or negative weight");
    DeviceGuard g(c->opts.device);
    int rc = eig_prepare(c, side);
    // the real-basis variant's Re rho pass runs over all of rho after the product: no split there
    const bool grouped = !c->real_basis;
    if (!rc) rc = density_matrix(c, side, nt, Q, (const cplx* const*)psi, w, (cplx*)rho, grouped);
    if (!rc) rc = eig_launch(c, side, (const cplx*)rho, evals, (cplx*)evecs, grouped && c->eig[side].ngroups == 2);
    return rc;
}

int tdmrg_hpsi_flops(tdmrg_ctx* c, int a, int b, double* flops) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!flops) return fail(c, TDMRG_EINVAL, "hpsi_flops: null output");
    if (!c->ham_set) return fail(c, TDMRG_ESTATE, "hpsi_flops: Hamiltonian not set");
    DeviceGuard g(c->opts.device);
    Plan* p = nullptr;
    int rc = get_plan(c, 0, -1, -1, a, b, a, b, &p);
    if (rc) return rc;
    *flops = p->flops;
    return TDMRG_OK;
}

namespace {
// polls a word that nothing sets; gives up after `spins` polls like every bounded wait of the library
__global__ void k_wait_probe(const volatile int* flag, int* status, long long spins) {
    if (threadIdx.x != 0) return;
    long long it = 0;
    while (*flag == 0) {
        if (++it > spins) {
            atomicOr(status, 4);
            break;
        }
    }
}
}  // namespace

int tdmrg_probe_wait(tdmrg_ctx* c, int64_t spins) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (spins < 1 || spins > (int64_t(1) << 26)) return fail(c, TDMRG_EINVAL, "probe_wait: spins must be in 1..2^26");
    DeviceGuard g(c->opts.device);
    int* flag = nullptr;
    int rc = dev_alloc(c, (void**)&flag, sizeof(int), "probe flag");
    if (rc) return rc;
    rc = cuda_check(c, cudaMemsetAsync(flag, 0, sizeof(int), c->stream), "probe flag");
    if (!rc) {
        k_wait_probe<<<1, 32, 0, c->stream>>>(flag, c->dstatus, (long long)spins);
        c->launches++;
        rc = cuda_check(c, cudaGetLastError(), "probe launch");
    }
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "probe wait");
    dev_free(c, flag, sizeof(int));
    return rc ? rc : check_device_status(c);
}

int tdmrg_set_orth_per_sm(tdmrg_ctx* c, int k) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (k < 0 || k > 8) return fail(c, TDMRG_EINVAL, "set_orth_per_sm: 0..8 blocks per SM");
    DeviceGuard g(c->opts.device);
    cudaStreamSynchronize(c->stream);
    c->orth_per_sm = k;
    drop_krylov(c);   // the Krylov workspaces are rebuilt with the new grid on their next use
    return TDMRG_OK;
}

int tdmrg_set_tile_m(tdmrg_ctx* c, int m) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (m != 0 && m != 64 && m != 128) return fail(c, TDMRG_EINVAL, "set_tile_m: m must be 0, 64 or 128");
    DeviceGuard g(c->opts.device);
    c->tile_m = m;
    drop_plans(c);   // plans are rebuilt with the new tile shape on their next use
    return TDMRG_OK;
}

int tdmrg_hpsi_tuning(tdmrg_ctx* c, int a, int b, int32_t* out) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!out) return fail(c, TDMRG_EINVAL, "hpsi_tuning: null output");
    if (!c->ham_set) return fail(c, TDMRG_ESTATE, "hpsi_tuning: Hamiltonian not set");
    DeviceGuard g(c->opts.device);
    Plan* p = nullptr;
    int rc = get_plan(c, 0, -1, -1, a, b, a, b, &p);
    if (rc) return rc;
    for (int s = 0; s < 2; ++s) {
        out[2 * s] = p->oz.ready ? p->oz.st[s].tmw : 0;
        out[2 * s + 1] = p->oz.ready ? p->oz.st[s].queue : -1;
    }
    return TDMRG_OK;
}

int tdmrg_set_schedule(tdmrg_ctx* c, int mode) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (mode < -1 || mode > 1) return fail(c, TDMRG_EINVAL, "set_schedule: mode must be -1, 0 or 1");
    DeviceGuard g(c->opts.device);
    c->schedule = mode;
    drop_plans(c);   // plans are rebuilt with the new schedule on their next use
    return TDMRG_OK;
}

int tdmrg_set_coefficients(tdmrg_ctx* c, const tdmrg_c64* coeff_d) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!c->ham_set) return fail(c, TDMRG_ESTATE, "set_coefficients: Hamiltonian not set");
    DeviceGuard g(c->opts.device);
    cudaStreamSynchronize(c->stream);
    c->dcoef = (const cplx*)coeff_d;
    drop_plans(c);   // plans are rebuilt with run-time coefficients on their next use
    return TDMRG_OK;
}

int tdmrg_set_real_basis(tdmrg_ctx* c, int on) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    c->real_basis = on ? 1 : 0;
    return TDMRG_OK;
}

int tdmrg_set_thin_dim(tdmrg_ctx* c, int dim) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (dim < 0 || dim > 64) return fail(c, TDMRG_EINVAL, "set_thin_dim: dim must be in 0..64");
    DeviceGuard g(c->opts.device);
    cudaStreamSynchronize(c->stream);
    c->thin_dim = dim;
    drop_plans(c);   // plans are rebuilt with the new split on their next use
    return TDMRG_OK;
}

int tdmrg_expect(tdmrg_ctx* c, int opL, int opR, int a, int b, const tdmrg_c64* psi, tdmrg_c64* out) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!psi || !out) return fail(c, TDMRG_EINVAL, "expect: null pointer");
    if (!c->side[0].set || !c->side[1].set) return fail(c, TDMRG_ESTATE, "expect: blocks not set");
    int64_t n = sector_size(c, a, b);
    if (n == 0) return fail(c, TDMRG_ESECTOR, "expect: empty sector");
    DeviceGuard g(c->opts.device);
    int rc = ensure_tmp(c, n);
    if (rc) return rc;
    rc = tdmrg_apply_op(c, opL, opR, a, b, psi, a, b, (tdmrg_c64*)c->tmp);
    if (rc) return rc;
    c->launches += 2;
    return cuda_check(c, launch_dot_final((const cplx*)psi, c->tmp, n, c->red, kRedBlocks, (cplx*)out, 1, c->stream),
                      "expect reduction");
}

int tdmrg_overlap_op(tdmrg_ctx* c, int opL, int opR, int a1, int b1, const tdmrg_c64* phi1, int a2, int b2,
                     const tdmrg_c64* phi2, tdmrg_c64* out) {
    if (check_ctx(c)) return TDMRG_EINVAL;
    if (!phi1 || !phi2 || !out) return fail(c, TDMRG_EINVAL, "overlap_op: null pointer");
    if (!c->side[0].set || !c->side[1].set) return fail(c, TDMRG_ESTATE, "overlap_op: blocks not set");
    const int64_t n1 = sector_size(c, a1, b1);
    if (n1 == 0 || sector_size(c, a2, b2) == 0) return fail(c, TDMRG_ESECTOR, "overlap_op: empty sector");
    DeviceGuard g(c->opts.device);
    if (opL < 0 && opR < 0) {   // both identities: the plain overlap <phi1|phi2>
        if (a1 != a2 || b1 != b2) return fail(c, TDMRG_ESECTOR, "overlap_op: identity between different sectors");
        c->launches += 1;
        return cuda_check(c, launch_dot_final((const cplx*)phi1, (const cplx*)phi2, n1, c->red, kRedBlocks, (cplx*)out, 0,
                                              c->stream), "overlap_op reduction");
    }
    int rc = ensure_tmp(c, n1);
    if (rc) return rc;
    rc = tdmrg_apply_op(c, opL, opR, a2, b2, phi2, a1, b1, (tdmrg_c64*)c->tmp);   // opL opR phi2, in Q1
    if (rc) return rc;
    c->launches += 2;
    return cuda_check(c, launch_dot_final((const cplx*)phi1, c->tmp, n1, c->red, kRedBlocks, (cplx*)out, 0, c->stream),
                      "overlap_op reduction");
}

}  // extern "C"
