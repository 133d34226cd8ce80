// Serving: continuous batching of time-evolution jobs on one GPU (declared in include/tdmrg.h).
//
// A server thread loops over: admit queued jobs in arrival order while the running jobs' footprint
// fits the HBM budget and a slot is free; for every running job whose step in flight has finished,
// record its observables and device time and enqueue the next step on the job's own stream; release
// finished and cancelled jobs.  A step is the time step of Sec. II.C: tdmrg_evolve (Krylov advance
// with n_v targets, the last target overwriting phi), tdmrg_density_eig (rho_L of the ground state + targets,
// weights of Sec. II.C, and its eigendecomposition) and one tdmrg_expect per observable.  The first step runs
// directly (it compiles the plans and allocates the workspace); the next steps replay a CUDA graph
// captured from one step.
//
// Batching (tdmrg_server_set_batching, max_group > 1): when jobs are admitted, the queued jobs that can
// share a time step (same precision, tau, n_v, n_K, number of steps and excitation sector shift; static
// coefficients; vector lengths within a factor of two) are admitted together, up to max_group, as one group.  A group runs on the direct sum
// of its members' superblocks: per time step one segmented Krylov advance (one grouped product per
// Lanczos step for every member), one grouped rho_L (every member normalised apart) and one
// eigendecomposition over every member's sectors, then each member's observables on its own context.
// Members finish together; a cancelled member stops recording at once and frees its slot with the group.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>

#include "internal.h"

namespace {

using namespace tdmrg;

struct Job {
    int64_t id = 0;
    std::chrono::steady_clock::time_point queued_at;
    int group = -1;                   // index of the group that runs this job (-1: runs alone)
    tdmrg_job d{};
    int status = TDMRG_JOB_QUEUED;
    bool cancel = false;
    std::string err;
    cudaStream_t stream = nullptr;
    cudaStream_t ctx_stream = nullptr;   // the context's stream before admission, restored at release
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool in_flight = false;
    int steps_done = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t n = 0, nrho = 0, nev = 0;
    cplx* phi = nullptr;
    std::vector<cplx*> targets;       // n_v - 1 own buffers, then phi
    cplx* rho = nullptr;
    cplx* evecs = nullptr;
    double* evals = nullptr;
    cplx* obs_d = nullptr;
    tdmrg_c64* obs_h = nullptr;       // pinned slot for the observables of the step in flight
    std::vector<tdmrg_c64> obs;       // steps x nobs
    std::vector<float> step_ms;
    size_t own_bytes = 0, footprint = 0;
    std::vector<double> times;
    double wgs = 0.0;
    std::vector<double> w;
};

struct Group {
    std::vector<int64_t> members;
    tdmrg_ctx* big = nullptr;
    int32_t qs[2] = {0, 0}, q0s[2] = {0, 0};
    std::vector<int64_t> off, off0, seg;
    int n_v = 0, nk = 0, steps = 0, nobs_max = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool in_flight = false, failed = false;
    int steps_done = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t n = 0, n0 = 0, nrho = 0, nev = 0;
    cplx* phi = nullptr;
    cplx* psi = nullptr;
    std::vector<cplx*> targets;       // n_v - 1 own buffers, then phi
    cplx* rho = nullptr;
    cplx* evecs = nullptr;
    double* evals = nullptr;
    cplx* obs_d = nullptr;            // 16 per member
    tdmrg_c64* obs_h = nullptr;
    std::vector<double> times;
    double wgs = 0.0;
    std::vector<double> w;
    size_t footprint = 0;
};

}  // namespace

struct tdmrg_server {
    int device = 0;
    size_t budget = 0;
    int max_active = 1;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    std::atomic<bool> stop{false};
    std::map<int64_t, std::unique_ptr<Job>> jobs;
    std::deque<int64_t> queue;
    std::vector<int64_t> active;
    int64_t next_id = 1;
    int max_group = 1;
    int window_us = 0;                 // how long the queue's front waits for partners before running alone
    std::map<int, std::unique_ptr<Group>> groups;
    int next_group = 0;
    int64_t grouped_jobs = 0;
    size_t in_use = 0;
    int finished = 0;
    std::string err = "no error";
};

namespace {

int job_fail(Job& j, const std::string& msg) {
    j.err = msg;
    j.status = TDMRG_JOB_FAILED;
    return TDMRG_ECUDA;
}

bool cuda_ok(Job& j, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return true;
    cudaGetLastError();
    job_fail(j, std::string(what) + ": " + cudaGetErrorString(e));
    return false;
}

// Enqueue one time step of the job on its stream (no host synchronisation; capturable).
int enqueue_step(Job& j) {
    tdmrg_ctx* c = j.d.ctx;
    int rc = tdmrg_evolve(c, j.d.q[0], j.d.q[1], (const tdmrg_c64*)j.phi, j.d.n_v, j.times.data(), j.d.nk,
                          (tdmrg_c64* const*)j.targets.data());
    if (rc) return rc;
    std::vector<int32_t> Q;
    std::vector<const tdmrg_c64*> ps;
    std::vector<double> ws;
    Q.push_back(j.d.q_gs[0]); Q.push_back(j.d.q_gs[1]); ps.push_back(j.d.psi_gs_d); ws.push_back(j.wgs);
    for (int x = 0; x < j.d.n_v; ++x) {
        Q.push_back(j.d.q[0]); Q.push_back(j.d.q[1]);
        ps.push_back((const tdmrg_c64*)j.targets[x]);
        ws.push_back(j.w[x]);
    }
    rc = tdmrg_density_eig(c, 0, (int)ps.size(), Q.data(), ps.data(), ws.data(), (tdmrg_c64*)j.rho, j.evals,
                           (tdmrg_c64*)j.evecs);
    if (rc) return rc;
    for (int k = 0; k < j.d.nobs; ++k) {
        rc = tdmrg_expect(c, j.d.obs_opL[k], j.d.obs_opR[k], j.d.q[0], j.d.q[1], (const tdmrg_c64*)j.phi,
                          (tdmrg_c64*)(j.obs_d + k));
        if (rc) return rc;
    }
    return TDMRG_OK;
}

size_t estimate(const Job& j) {
    // operators and plans already in the context, plus Krylov vectors, stage-1 intermediates (about
    // one vector per term), targets, rho_L and the eigensolver workspace
    const size_t vec = (size_t)j.n * sizeof(cplx);
    return j.d.ctx->allocated + (size_t)(j.d.nk + j.d.n_v + 12) * vec + (size_t)10 * j.nrho * sizeof(cplx);
}

void release_job(Job& j) {
    if (j.stream) cudaStreamSynchronize(j.stream);
    if (j.stream && j.d.ctx && j.d.ctx->stream == j.stream) tdmrg_set_stream(j.d.ctx, (void*)j.ctx_stream);
    if (j.exec) cudaGraphExecDestroy(j.exec);
    j.exec = nullptr;
    for (size_t x = 0; x + 1 < j.targets.size(); ++x) cudaFree(j.targets[x]);
    j.targets.clear();
    cudaFree(j.phi); cudaFree(j.rho); cudaFree(j.evecs); cudaFree(j.evals); cudaFree(j.obs_d);
    j.phi = nullptr; j.rho = nullptr; j.evecs = nullptr; j.evals = nullptr; j.obs_d = nullptr;
    if (j.obs_h) cudaFreeHost(j.obs_h);
    j.obs_h = nullptr;
    if (j.ev0) cudaEventDestroy(j.ev0);
    if (j.ev1) cudaEventDestroy(j.ev1);
    j.ev0 = j.ev1 = nullptr;
    if (j.stream) cudaStreamDestroy(j.stream);
    j.stream = nullptr;
}

bool admit(tdmrg_server* s, Job& j) {
    tdmrg_ctx* c = j.d.ctx;
    j.times.resize(j.d.n_v);
    for (int x = 0; x < j.d.n_v; ++x) j.times[x] = x * j.d.tau / (j.d.n_v - 1);
    j.w.resize(j.d.n_v);
    tdmrg_tst_weights(j.d.n_v, &j.wgs, j.w.data());
    if (!cuda_ok(j, cudaStreamCreateWithFlags(&j.stream, cudaStreamNonBlocking), "job stream")) return false;
    if (!cuda_ok(j, cudaEventCreate(&j.ev0), "job event") || !cuda_ok(j, cudaEventCreate(&j.ev1), "job event")) return false;
    j.ctx_stream = c->stream;
    cudaStreamSynchronize(j.ctx_stream);   // work the caller queued on the context (e.g. loading) is done
    tdmrg_set_stream(c, j.stream);
    size_t vb = (size_t)j.n * sizeof(cplx);
    j.targets.assign(j.d.n_v, nullptr);
    bool ok = cuda_ok(j, cudaMalloc(&j.phi, vb), "job buffers");
    for (int x = 0; ok && x + 1 < j.d.n_v; ++x) ok = cuda_ok(j, cudaMalloc(&j.targets[x], vb), "job buffers");
    if (ok) ok = cuda_ok(j, cudaMalloc(&j.rho, j.nrho * sizeof(cplx)), "job buffers");
    if (ok) ok = cuda_ok(j, cudaMalloc(&j.evecs, j.nrho * sizeof(cplx)), "job buffers");
    if (ok) ok = cuda_ok(j, cudaMalloc(&j.evals, j.nev * sizeof(double)), "job buffers");
    if (ok) ok = cuda_ok(j, cudaMalloc(&j.obs_d, 16 * sizeof(cplx)), "job buffers");
    if (ok) ok = cuda_ok(j, cudaMallocHost(&j.obs_h, 16 * sizeof(tdmrg_c64)), "job buffers");
    if (!ok) return false;
    j.targets[j.d.n_v - 1] = j.phi;
    j.own_bytes = (size_t)j.d.n_v * vb + 2 * j.nrho * sizeof(cplx) + j.nev * sizeof(double) + 16 * sizeof(cplx);
    if (!cuda_ok(j, cudaMemcpyAsync(j.phi, j.d.phi0_d, vb, cudaMemcpyDeviceToDevice, j.stream), "job phi0")) return false;
    j.status = TDMRG_JOB_RUNNING;
    (void)s;
    return true;
}

bool launch_step(Job& j) {
    tdmrg_ctx* c = j.d.ctx;
    if (!cuda_ok(j, cudaEventRecord(j.ev0, j.stream), "step event")) return false;
    if (j.steps_done == 0) {
        int rc = enqueue_step(j);   // direct: compiles plans, allocates workspace
        if (rc) { job_fail(j, tdmrg_last_error(c)); return false; }
    } else {
        if (!j.exec) {
            cudaGraph_t g = nullptr;
            if (!cuda_ok(j, cudaStreamBeginCapture(j.stream, cudaStreamCaptureModeThreadLocal), "graph capture")) return false;
            int rc = enqueue_step(j);
            cudaError_t e = cudaStreamEndCapture(j.stream, &g);
            if (rc) { if (g) cudaGraphDestroy(g); job_fail(j, tdmrg_last_error(c)); return false; }
            if (!cuda_ok(j, e, "graph capture")) return false;
            e = cudaGraphInstantiate(&j.exec, g, 0);
            cudaGraphDestroy(g);
            if (!cuda_ok(j, e, "graph instantiate")) return false;
        }
        if (!cuda_ok(j, cudaGraphLaunch(j.exec, j.stream), "graph launch")) return false;
    }
    if (j.d.nobs > 0 &&
        !cuda_ok(j, cudaMemcpyAsync(j.obs_h, j.obs_d, j.d.nobs * sizeof(tdmrg_c64), cudaMemcpyDeviceToHost, j.stream),
                 "observables"))
        return false;
    if (!cuda_ok(j, cudaEventRecord(j.ev1, j.stream), "step event")) return false;
    j.in_flight = true;
    return true;
}

bool compatible(const Job& a, const Job& b) {
    const tdmrg_ctx* x = a.d.ctx;
    const tdmrg_ctx* y = b.d.ctx;
    return x->opts.prec == y->opts.prec && x->opts.ozaki_slices == y->opts.ozaki_slices && a.d.tau == b.d.tau &&
           a.d.n_v == b.d.n_v && a.d.nk == b.d.nk && a.d.steps == b.d.steps && !x->dcoef && !y->dcoef &&
           a.d.q[0] - a.d.q_gs[0] == b.d.q[0] - b.d.q_gs[0] && a.d.q[1] - a.d.q_gs[1] == b.d.q[1] - b.d.q_gs[1] &&
           x->opts.nk_max >= b.d.nk && x != y &&
           // similar sizes: a group's step lasts as long as its largest member's
           std::max(a.n, b.n) <= 2 * std::min(a.n, b.n);
}

void release_group(tdmrg_server* s, Group& g) {
    if (g.stream) cudaStreamSynchronize(g.stream);
    for (int64_t id : g.members) {
        Job& j = *s->jobs[id];
        if (j.d.ctx) tdmrg_set_stream(j.d.ctx, (void*)j.ctx_stream);   // the legacy default stream is null
    }
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    for (size_t x = 0; x + 1 < g.targets.size(); ++x) cudaFree(g.targets[x]);
    g.targets.clear();
    cudaFree(g.phi); cudaFree(g.psi); cudaFree(g.rho); cudaFree(g.evecs); cudaFree(g.evals); cudaFree(g.obs_d);
    g.phi = g.psi = g.rho = g.evecs = g.obs_d = nullptr;
    g.evals = nullptr;
    if (g.obs_h) cudaFreeHost(g.obs_h);
    g.obs_h = nullptr;
    if (g.big) tdmrg_destroy(g.big);
    g.big = nullptr;
    if (g.ev0) cudaEventDestroy(g.ev0);
    if (g.ev1) cudaEventDestroy(g.ev1);
    g.ev0 = g.ev1 = nullptr;
    if (g.stream) cudaStreamDestroy(g.stream);
    g.stream = nullptr;
}

// The group's direct sum, buffers and the members' start vectors.
bool admit_group(tdmrg_server* s, Group& g) {
    Job& j0 = *s->jobs[g.members[0]];
    auto gfail = [&](const std::string& m) {
        for (int64_t id : g.members) job_fail(*s->jobs[id], m);
        g.failed = true;
        return false;
    };
    if (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&g.ev0) != cudaSuccess ||
        cudaEventCreate(&g.ev1) != cudaSuccess) {
        cudaGetLastError();
        return gfail("group stream");
    }
    tdmrg_opts o = j0.d.ctx->opts;
    o.stream = g.stream;
    o.hbm_budget = 0;
    if (tdmrg_create(&g.big, &o)) return gfail("group context: " + std::string(tdmrg_last_error(nullptr)));
    std::vector<tdmrg_ctx*> ctxs;
    std::vector<int32_t> Q;
    for (int64_t id : g.members) {
        Job& j = *s->jobs[id];
        j.ctx_stream = j.d.ctx->stream;
        cudaStreamSynchronize(j.ctx_stream);   // work the caller queued on the context is done
        ctxs.push_back(j.d.ctx);
        Q.push_back(j.d.q[0]);
        Q.push_back(j.d.q[1]);
    }
    g.off.assign(g.members.size() + 1, 0);
    if (tdmrg_direct_sum(g.big, (int)ctxs.size(), ctxs.data(), Q.data(), g.qs, g.off.data()))
        return gfail("group direct sum: " + std::string(tdmrg_last_error(g.big)));
    g.q0s[0] = g.qs[0] - (j0.d.q[0] - j0.d.q_gs[0]);
    g.q0s[1] = g.qs[1] - (j0.d.q[1] - j0.d.q_gs[1]);
    g.off0.assign(g.members.size() + 1, 0);
    for (size_t k = 0; k < g.members.size(); ++k) {
        Job& j = *s->jobs[g.members[k]];
        g.off0[k + 1] = g.off0[k] + sector_size(j.d.ctx, j.d.q_gs[0], j.d.q_gs[1]);
        g.seg.push_back(g.off[k + 1] - g.off[k]);
        tdmrg_set_stream(j.d.ctx, g.stream);
        g.nobs_max = std::max(g.nobs_max, j.d.nobs);
    }
    g.n = g.off.back();
    g.n0 = g.off0.back();
    if (sector_size(g.big, g.q0s[0], g.q0s[1]) != g.n0) return gfail("group: ground-state sectors do not add up");
    for (int dd : g.big->side[0].dim) { g.nrho += (int64_t)dd * dd; g.nev += dd; }
    g.n_v = j0.d.n_v; g.nk = j0.d.nk; g.steps = j0.d.steps;
    g.times.resize(g.n_v);
    for (int x = 0; x < g.n_v; ++x) g.times[x] = x * j0.d.tau / (g.n_v - 1);
    g.w.resize(g.n_v);
    tdmrg_tst_weights(g.n_v, &g.wgs, g.w.data());
    const size_t vb = (size_t)g.n * sizeof(cplx), m = g.members.size();
    g.targets.assign(g.n_v, nullptr);
    bool ok = cudaMalloc(&g.phi, vb) == cudaSuccess && cudaMalloc(&g.psi, (size_t)g.n0 * sizeof(cplx)) == cudaSuccess;
    for (int x = 0; ok && x + 1 < g.n_v; ++x) ok = cudaMalloc(&g.targets[x], vb) == cudaSuccess;
    if (ok) ok = cudaMalloc(&g.rho, g.nrho * sizeof(cplx)) == cudaSuccess && cudaMalloc(&g.evecs, g.nrho * sizeof(cplx)) == cudaSuccess &&
                 cudaMalloc(&g.evals, g.nev * sizeof(double)) == cudaSuccess &&
                 cudaMalloc(&g.obs_d, 16 * m * sizeof(cplx)) == cudaSuccess &&
                 cudaMallocHost(&g.obs_h, 16 * m * sizeof(tdmrg_c64)) == cudaSuccess;
    if (!ok) { cudaGetLastError(); return gfail("group buffers"); }
    g.targets[g.n_v - 1] = g.phi;
    for (size_t k = 0; k < m && ok; ++k) {
        Job& j = *s->jobs[g.members[k]];
        ok = cudaMemcpyAsync(g.phi + g.off[k], j.d.phi0_d, (size_t)g.seg[k] * sizeof(cplx), cudaMemcpyDeviceToDevice, g.stream) ==
                 cudaSuccess &&
             cudaMemcpyAsync(g.psi + g.off0[k], j.d.psi_gs_d, (size_t)(g.off0[k + 1] - g.off0[k]) * sizeof(cplx),
                             cudaMemcpyDeviceToDevice, g.stream) == cudaSuccess;
        j.status = TDMRG_JOB_RUNNING;
    }
    if (!ok) { cudaGetLastError(); return gfail("group start vectors"); }
    return true;
}

// One time step of every member (capturable).
int enqueue_group_step(tdmrg_server* s, Group& g) {
    int rc = tdmrg_evolve_segments(g.big, g.qs[0], g.qs[1], (const tdmrg_c64*)g.phi, (int)g.seg.size(), g.seg.data(), g.n_v,
                                   g.times.data(), g.nk, (tdmrg_c64* const*)g.targets.data());
    if (rc) return rc;
    std::vector<int32_t> Q = {g.q0s[0], g.q0s[1]};
    std::vector<const tdmrg_c64*> ps = {(const tdmrg_c64*)g.psi};
    std::vector<double> ws = {g.wgs};
    for (int x = 0; x < g.n_v; ++x) {
        Q.push_back(g.qs[0]); Q.push_back(g.qs[1]);
        ps.push_back((const tdmrg_c64*)g.targets[x]);
        ws.push_back(g.w[x]);
    }
    rc = tdmrg_density_eig(g.big, 0, (int)ps.size(), Q.data(), ps.data(), ws.data(), (tdmrg_c64*)g.rho, g.evals,
                           (tdmrg_c64*)g.evecs);
    if (rc) return rc;
    for (size_t k = 0; k < g.members.size(); ++k) {
        Job& j = *s->jobs[g.members[k]];
        for (int o = 0; o < j.d.nobs; ++o) {
            rc = tdmrg_expect(j.d.ctx, j.d.obs_opL[o], j.d.obs_opR[o], j.d.q[0], j.d.q[1], (const tdmrg_c64*)(g.phi + g.off[k]),
                              (tdmrg_c64*)(g.obs_d + 16 * k + o));
            if (rc) return rc;
        }
    }
    return TDMRG_OK;
}

bool launch_group_step(tdmrg_server* s, Group& g) {
    auto gfail = [&](const std::string& m) {
        for (int64_t id : g.members) if (s->jobs[id]->status == TDMRG_JOB_RUNNING) job_fail(*s->jobs[id], m);
        g.failed = true;
        return false;
    };
    if (cudaEventRecord(g.ev0, g.stream) != cudaSuccess) { cudaGetLastError(); return gfail("group event"); }
    if (g.steps_done == 0) {
        if (enqueue_group_step(s, g)) return gfail(tdmrg_last_error(g.big));
    } else {
        if (!g.exec) {
            cudaGraph_t gr = nullptr;
            if (cudaStreamBeginCapture(g.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                cudaGetLastError();
                return gfail("group graph capture");
            }
            const int rc = enqueue_group_step(s, g);
            cudaError_t e = cudaStreamEndCapture(g.stream, &gr);
            if (rc || e != cudaSuccess) { if (gr) cudaGraphDestroy(gr); cudaGetLastError(); return gfail("group graph capture"); }
            e = cudaGraphInstantiate(&g.exec, gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) { cudaGetLastError(); return gfail("group graph instantiate"); }
        }
        if (cudaGraphLaunch(g.exec, g.stream) != cudaSuccess) { cudaGetLastError(); return gfail("group graph launch"); }
    }
    if (g.nobs_max > 0 && cudaMemcpyAsync(g.obs_h, g.obs_d, 16 * g.members.size() * sizeof(tdmrg_c64),
                                          cudaMemcpyDeviceToHost, g.stream) != cudaSuccess) {
        cudaGetLastError();
        return gfail("group observables");
    }
    if (cudaEventRecord(g.ev1, g.stream) != cudaSuccess) { cudaGetLastError(); return gfail("group event"); }
    g.in_flight = true;
    return true;
}

// Admission of a group: the queue's front job and the compatible queued jobs after it.  GROUP_WAIT: the
// front has no partner yet and is younger than the batching window.
enum { GROUP_NONE = 0, GROUP_ADMITTED = 1, GROUP_WAIT = 2 };
int try_group(tdmrg_server* s) {
    if (s->max_group < 2 || s->queue.empty()) return GROUP_NONE;
    Job& j0 = *s->jobs[s->queue.front()];
    if (j0.cancel) return GROUP_NONE;
    const int room = s->max_active - (int)s->active.size();
    std::vector<int64_t> pick = {j0.id};
    for (size_t i = 1; i < s->queue.size() && (int)pick.size() < std::min(s->max_group, room); ++i) {
        Job& j = *s->jobs[s->queue[i]];
        if (!j.cancel && compatible(j0, j)) pick.push_back(j.id);
    }
    if (pick.size() < 2) {
        const auto age = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - j0.queued_at);
        return age.count() < s->window_us && room >= 2 ? GROUP_WAIT : GROUP_NONE;
    }
    size_t est = 0;
    for (int64_t id : pick) est += 2 * estimate(*s->jobs[id]);   // the members' copies in the direct sum as well
    if (s->budget && !s->active.empty() && s->in_use + est > s->budget) return GROUP_NONE;
    for (int64_t id : pick) s->queue.erase(std::find(s->queue.begin(), s->queue.end(), id));
    const int gid = s->next_group++;
    std::unique_ptr<Group> g(new Group());
    g->members = pick;
    g->footprint = est;
    for (int64_t id : pick) { s->jobs[id]->group = gid; s->active.push_back(id); }
    s->grouped_jobs += (int64_t)pick.size();
    s->in_use += est;
    Group& gr = *g;
    s->groups[gid] = std::move(g);
    if (!admit_group(s, gr)) gr.failed = true;
    return GROUP_ADMITTED;
}

// Progress of the running groups; returns true if anything changed.
bool pass_groups(tdmrg_server* s) {
    bool progress = false;
    for (auto it = s->groups.begin(); it != s->groups.end();) {
        Group& g = *it->second;
        bool done = g.failed;
        if (!done && g.in_flight) {
            const cudaError_t q = cudaEventQuery(g.ev1);
            if (q == cudaErrorNotReady) { ++it; continue; }
            g.in_flight = false;
            progress = true;
            if (q != cudaSuccess) {
                cudaGetLastError();
                for (int64_t id : g.members) job_fail(*s->jobs[id], std::string("group step: ") + cudaGetErrorString(q));
                done = true;
            } else {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, g.ev0, g.ev1);
                g.steps_done++;
                for (size_t k = 0; k < g.members.size(); ++k) {
                    Job& j = *s->jobs[g.members[k]];
                    if (j.status != TDMRG_JOB_RUNNING) continue;
                    j.step_ms.push_back(ms);
                    for (int o = 0; o < j.d.nobs; ++o) j.obs.push_back(g.obs_h[16 * k + o]);
                    j.steps_done = g.steps_done;
                    if (j.cancel) j.status = TDMRG_JOB_CANCELLED;
                    else if (j.steps_done >= j.d.steps) j.status = TDMRG_JOB_DONE;
                }
                if (g.steps_done == 1) {   // plans and workspace exist now: the real footprint
                    size_t real = g.big->allocated + (size_t)(g.n_v + 1) * g.n * sizeof(cplx) + 2 * g.nrho * sizeof(cplx);
                    for (int64_t id : g.members) real += s->jobs[id]->d.ctx->allocated;
                    s->in_use = s->in_use - std::min(s->in_use, g.footprint) + real;
                    g.footprint = real;
                }
                if (g.steps_done >= g.steps) done = true;
            }
        }
        bool all_cancelled = true;
        for (int64_t id : g.members) all_cancelled &= s->jobs[id]->cancel;
        if (!done && all_cancelled) done = true;
        if (!done && !g.in_flight) {
            progress = true;
            if (!launch_group_step(s, g)) done = true;
        }
        if (done) {
            release_group(s, g);
            for (int64_t id : g.members) {
                Job& j = *s->jobs[id];
                if (j.status == TDMRG_JOB_RUNNING) j.status = j.cancel ? TDMRG_JOB_CANCELLED : TDMRG_JOB_FAILED;
                s->finished++;
                s->active.erase(std::find(s->active.begin(), s->active.end(), id));
            }
            s->in_use -= std::min(s->in_use, g.footprint);
            it = s->groups.erase(it);
            continue;
        }
        ++it;
    }
    return progress;
}

// One pass of the server loop.  Returns true if anything changed.
bool pass(tdmrg_server* s) {
    bool progress = false;
    std::unique_lock<std::mutex> lk(s->mu);
    // admission in arrival order (a group first, when batching is on and the queue holds one)
    while (!s->queue.empty() && (int)s->active.size() < s->max_active) {
        const int tg = try_group(s);
        if (tg == GROUP_ADMITTED) { progress = true; continue; }
        if (tg == GROUP_WAIT) break;
        Job& j = *s->jobs[s->queue.front()];
        if (j.cancel) {
            j.status = TDMRG_JOB_CANCELLED;
            s->finished++;
            s->queue.pop_front();
            progress = true;
            continue;
        }
        const size_t est = estimate(j);
        if (s->budget && !s->active.empty() && s->in_use + est > s->budget) break;
        s->queue.pop_front();
        progress = true;
        if (!admit(s, j)) {
            release_job(j);
            s->finished++;
            continue;
        }
        j.footprint = est;
        s->in_use += est;
        s->active.push_back(j.id);
    }
    progress |= pass_groups(s);
    // progress of running jobs
    for (size_t a = 0; a < s->active.size();) {
        Job& j = *s->jobs[s->active[a]];
        if (j.group >= 0) { ++a; continue; }   // driven by its group
        bool done = false;
        if (j.in_flight) {
            cudaError_t q = cudaEventQuery(j.ev1);
            if (q == cudaErrorNotReady) { ++a; continue; }
            j.in_flight = false;
            progress = true;
            if (!cuda_ok(j, q, "job step")) {
                done = true;
            } else {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, j.ev0, j.ev1);
                j.step_ms.push_back(ms);
                for (int k = 0; k < j.d.nobs; ++k) j.obs.push_back(j.obs_h[k]);
                j.steps_done++;
                if (j.steps_done == 1) {   // the plans and workspace exist now: use the real footprint
                    const size_t real = j.d.ctx->allocated + j.own_bytes;
                    s->in_use = s->in_use - j.footprint + real;
                    j.footprint = real;
                }
                if (j.steps_done >= j.d.steps) { j.status = TDMRG_JOB_DONE; done = true; }
            }
        }
        if (!done && j.cancel) { j.status = TDMRG_JOB_CANCELLED; done = true; }
        if (!done && !j.in_flight) {
            progress = true;
            if (!launch_step(j)) done = true;
        }
        if (done) {
            release_job(j);
            s->in_use -= std::min(s->in_use, j.footprint);
            s->finished++;
            s->active.erase(s->active.begin() + a);
            continue;
        }
        ++a;
    }
    return progress;
}

void worker(tdmrg_server* s) {
    cudaSetDevice(s->device);
    while (!s->stop.load()) {
        if (!pass(s)) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

int sfail(tdmrg_server* s, int code, const std::string& msg) {
    if (s) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->err = msg;
    }
    return fail(nullptr, code, msg);
}

}  // namespace

extern "C" {

int tdmrg_server_create(tdmrg_server** out, int device, size_t budget, int max_active) {
    if (!out || max_active < 1) return fail(nullptr, TDMRG_EINVAL, "server_create: bad argument");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(nullptr, TDMRG_ECUDA, "server_create: no CUDA device " + std::to_string(device));
    }
    tdmrg_server* s = new (std::nothrow) tdmrg_server();
    if (!s) return fail(nullptr, TDMRG_ENOMEM, "host allocation");
    s->device = device;
    s->budget = budget;
    s->max_active = max_active;
    s->worker = std::thread(worker, s);
    *out = s;
    return TDMRG_OK;
}

int tdmrg_server_set_batching(tdmrg_server* s, int max_group, int window_us) {
    if (!s || max_group < 1 || window_us < 0) return fail(nullptr, TDMRG_EINVAL, "server_set_batching: bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    s->max_group = max_group;
    s->window_us = window_us;
    return TDMRG_OK;
}

int tdmrg_server_batch_stats(tdmrg_server* s, int* groups, int64_t* grouped_jobs) {
    if (!s) return fail(nullptr, TDMRG_EINVAL, "server_batch_stats: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (groups) *groups = s->next_group;
    if (grouped_jobs) *grouped_jobs = s->grouped_jobs;
    return TDMRG_OK;
}

int tdmrg_server_submit(tdmrg_server* s, const tdmrg_job* job, int64_t* id) {
    if (!s || !job || !id) return sfail(s, TDMRG_EINVAL, "server_submit: null argument");
    const tdmrg_job& d = *job;
    // rho_L takes the ground state and the n_v targets: at most 12 states
    if (!d.ctx || !d.psi_gs_d || !d.phi0_d || d.n_v < 2 || d.n_v > 11 || d.nk < 1 || d.nk > d.ctx->opts.nk_max ||
        d.steps < 1 || d.nobs < 0 || d.nobs > 16 || !(d.tau > 0.0))
        return sfail(s, TDMRG_EINVAL, "server_submit: bad job description");
    if (d.ctx->opts.device != s->device) return sfail(s, TDMRG_EINVAL, "server_submit: context on another device");
    if (!d.ctx->ham_set) return sfail(s, TDMRG_ESTATE, "server_submit: Hamiltonian not set");
    std::unique_ptr<Job> j(new Job());
    j->d = d;
    j->n = sector_size(d.ctx, d.q[0], d.q[1]);
    for (int dd : d.ctx->side[0].dim) { j->nrho += (int64_t)dd * dd; j->nev += dd; }
    if (j->n == 0) return sfail(s, TDMRG_ESECTOR, "server_submit: empty sector");
    std::lock_guard<std::mutex> lk(s->mu);
    j->id = s->next_id++;
    j->queued_at = std::chrono::steady_clock::now();
    *id = j->id;
    s->queue.push_back(j->id);
    s->jobs[j->id] = std::move(j);
    s->cv.notify_all();
    return TDMRG_OK;
}

int tdmrg_server_poll(tdmrg_server* s, int64_t id, int* status, int* steps_done, tdmrg_c64* obs, float* step_ms) {
    if (!s) return fail(nullptr, TDMRG_EINVAL, "server_poll: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) {
        s->err = "server_poll: unknown job";
        return TDMRG_EINVAL;
    }
    const Job& j = *it->second;
    if (status) *status = j.status;
    if (steps_done) *steps_done = j.steps_done;
    if (obs && !j.obs.empty()) memcpy(obs, j.obs.data(), j.obs.size() * sizeof(tdmrg_c64));
    if (step_ms && !j.step_ms.empty()) memcpy(step_ms, j.step_ms.data(), j.step_ms.size() * sizeof(float));
    return TDMRG_OK;
}

int tdmrg_server_cancel(tdmrg_server* s, int64_t id) {
    if (!s) return fail(nullptr, TDMRG_EINVAL, "server_cancel: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) {
        s->err = "server_cancel: unknown job";
        return TDMRG_EINVAL;
    }
    it->second->cancel = true;
    s->cv.notify_all();
    return TDMRG_OK;
}

int tdmrg_server_stats(tdmrg_server* s, int* queued, int* running, int* finished, size_t* bytes) {
    if (!s) return fail(nullptr, TDMRG_EINVAL, "server_stats: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int)s->queue.size();
    if (running) *running = (int)s->active.size();
    if (finished) *finished = s->finished;
    if (bytes) *bytes = s->in_use;
    return TDMRG_OK;
}

int tdmrg_server_destroy(tdmrg_server* s) {
    if (!s) return TDMRG_OK;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (auto& kv : s->groups) release_group(s, *kv.second);
    for (auto& kv : s->jobs) if (kv.second->group < 0) release_job(*kv.second);
    delete s;
    return TDMRG_OK;
}

const char* tdmrg_server_last_error(tdmrg_server* s, int64_t id) {
    if (!s) return "null server";
    std::lock_guard<std::mutex> lk(s->mu);
    if (id >= 0) {
        auto it = s->jobs.find(id);
        if (it != s->jobs.end()) return it->second->err.c_str();
    }
    return s->err.c_str();
}

}  // extern "C"
