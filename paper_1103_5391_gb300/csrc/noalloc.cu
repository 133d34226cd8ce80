// H psi for callers that cannot allocate device memory while they run.
//
// Some callers may not call cudaMalloc (or any allocator) once they are running: a real-time or
// latency-critical loop that forbids allocation after initialisation, a host framework whose own
// memory pool owns all device memory, or a plugin that may only touch buffers handed to it.
// tdmrg_apply_h_static serves them: it runs the same grouped sector-pair GEMM as tdmrg_apply_h,
// but every byte of scratch it needs (the stage-1 intermediates Psi_{q'} B^T, the split-K partial
// tiles and their completion tickets) lives in the file-scope device array below, which the CUDA
// runtime creates when the library's module is loaded.  The call itself allocates nothing.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB, held on every device that loads the library

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void* g_static_ptr[128] = {nullptr};

// Device address of the static array for `dev` (the current device).  In host code the array's
// name is only a host-side stand-in, so the address must come from cudaGetSymbolAddress, once per
// device, with that device current.
int static_scratch(tdmrg_ctx* c, int dev, void** out) {
    if (dev < 0 || dev >= 128) return tdmrg::fail(c, TDMRG_EINVAL, "apply_h_static: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return tdmrg::fail(c, TDMRG_ECUDA, std::string("apply_h_static: cudaGetSymbolAddress failed: ") +
                                                   cudaGetErrorString(e));
        }
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return TDMRG_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int tdmrg_apply_h_static(tdmrg_ctx* c, int n_up, int n_dn, const tdmrg_c64* psi, tdmrg_c64* out) {
    using namespace tdmrg;
    if (!c) return fail(nullptr, TDMRG_EINVAL, "null context");
    if (!psi || !out) return fail(c, TDMRG_EINVAL, "apply_h_static: null vector");
    if (!c->ham_set) return fail(c, TDMRG_ESTATE, "apply_h_static: Hamiltonian not set");
    auto it = c->plans.find(std::make_tuple(0, -1, -1, n_up, n_dn, n_up, n_dn));
    if (it == c->plans.end())
        return fail(c, TDMRG_ESTATE,
                    "apply_h_static: sector not prepared; call tdmrg_apply_h or tdmrg_hpsi_flops for this sector "
                    "once during set-up");
    const Plan& p = *it->second;
    if (p.n_in == 0) return TDMRG_OK;
    // layout of the static array: intermediates | partials (stage 1, 2) | tickets (stage 1, 2)
    const size_t tile = (size_t)kTileF64 * kTileF64 * sizeof(cplx);
    const size_t off_p1 = align256((size_t)p.scratch * sizeof(cplx));
    const size_t off_p2 = off_p1 + align256((size_t)p.stage1.npartial * tile);
    const size_t off_c1 = off_p2 + align256((size_t)p.stage2.npartial * tile);
    const size_t off_c2 = off_c1 + align256((size_t)p.stage1.nsplit * sizeof(int));
    const size_t need = off_c2 + align256((size_t)p.stage2.nsplit * sizeof(int));
    if (need > kStaticScratchBytes)
        return fail(c, TDMRG_ENOMEM, "apply_h_static: sector needs " + std::to_string(need) +
                                         " bytes of scratch, above the static limit of " +
                                         std::to_string(kStaticScratchBytes) + " bytes (32 MiB)");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->opts.device && cudaSetDevice(c->opts.device) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, TDMRG_ECUDA, "apply_h_static: cannot select the context's device");
    }
    unsigned char* base = nullptr;
    int rc = static_scratch(c, c->opts.device, (void**)&base);
    // the completion tickets must start at zero (the array keeps the previous call's contents)
    if (!rc && need > off_c1)
        rc = cuda_check(c, cudaMemsetAsync(base + off_c1, 0, need - off_c1, c->stream), "apply_h_static ticket reset");
    GemmArgs a{};
    a.bufs[BUF_OPS] = c->pool;
    a.bufs[BUF_IN] = (cplx*)psi;
    a.bufs[BUF_SCRATCH] = (cplx*)base;
    a.bufs[BUF_OUT] = (cplx*)out;
    a.dscale = c->dscale;
    a.dcoef = c->dcoef;
    for (int st = 0; st < 2 && !rc; ++st) {
        const TaskList& tl = st == 0 ? p.stage1 : p.stage2;
        if (tl.tiles.empty()) continue;
        a.tasks = tl.d_tasks; a.segs = tl.d_segs; a.tiles = tl.d_tiles; a.ntiles = (int)tl.tiles.size();
        a.partials = (cplx*)(base + (st == 0 ? off_p1 : off_p2));
        a.counters = (int*)(base + (st == 0 ? off_c1 : off_c2));
        rc = cuda_check(c, launch_gemm_f64(a, c->stream, nullptr, 0), "apply_h_static launch");
        c->launches++;
    }
    if (prev >= 0 && prev != c->opts.device) cudaSetDevice(prev);
    return rc;
}
