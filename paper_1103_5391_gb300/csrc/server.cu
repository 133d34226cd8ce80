// Serving: continuous batching of time-evolution jobs on one GPU (declared in include/tdmrg.h).
//
// A server thread loops over: admit queued jobs in arrival order while the running jobs' footprint
// fits the HBM budget and a slot is free; for every running job whose step in flight has finished,
// record its observables and device time and enqueue the next step on the job's own stream; release
// finished and cancelled jobs.  A step is the time step of Sec. II.C: tdmrg_evolve (Krylov advance
// with n_v targets, the last target overwriting phi), tdmrg_density_matrix (ground state + targets,
// weights of Sec. II.C), tdmrg_rho_eig and one tdmrg_expect per observable.  The first step runs
// directly (it compiles the plans and allocates the workspace); the next steps replay a CUDA graph
// captured from one step.
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
    rc = tdmrg_density_matrix(c, (int)ps.size(), Q.data(), ps.data(), ws.data(), (tdmrg_c64*)j.rho);
    if (rc) return rc;
    rc = tdmrg_rho_eig(c, (const tdmrg_c64*)j.rho, j.evals, (tdmrg_c64*)j.evecs);
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

// One pass of the server loop.  Returns true if anything changed.
bool pass(tdmrg_server* s) {
    bool progress = false;
    std::unique_lock<std::mutex> lk(s->mu);
    // admission in arrival order
    while (!s->queue.empty() && (int)s->active.size() < s->max_active) {
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
    // progress of running jobs
    for (size_t a = 0; a < s->active.size();) {
        Job& j = *s->jobs[s->active[a]];
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
    for (auto& kv : s->jobs) release_job(*kv.second);
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
