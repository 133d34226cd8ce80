// Measurement entry points (include/tdmrg_bench.h): launch counter, flop count of a compiled H psi,
// and the device's sustained FP64 throughput.
#include "../../include/tdmrg_bench.h"
#include "internal.h"

namespace {

constexpr int kIters = 2048;

__global__ void __launch_bounds__(256) k_dmma_peak(double* out, double seed) {
    // four independent accumulation chains with distinct operands, so none can be merged
    double a[4], b[4], c[4][2];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = seed + threadIdx.x * 1e-3 + r * 0.125;
        b[r] = 1.0 + threadIdx.x * 1e-4 - r * 0.0625;
        c[r][0] = r;
        c[r][1] = -r;
    }
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                         : "+d"(c[r][0]), "+d"(c[r][1]) : "d"(a[r]), "d"(b[r]));
    }
    double s = 0.0;
    for (int r = 0; r < 4; ++r) s += c[r][0] + c[r][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_dfma_peak(double* out, double a, double b) {
    double x[8];
    for (int r = 0; r < 8; ++r) x[r] = threadIdx.x + r;
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r) x[r] = fma(x[r], a, b);
    }
    double s = 0.0;
    for (int r = 0; r < 8; ++r) s += x[r];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

int tdmrg_launch_count(tdmrg_ctx* c, int64_t* count) {
    if (!c || !count) return tdmrg::fail(c, TDMRG_EINVAL, "launch_count: null argument");
    *count = c->launches;
    return TDMRG_OK;
}

int tdmrg_alloc_count(tdmrg_ctx* c, int64_t* count, int64_t* bytes) {
    if (!c || !count || !bytes) return tdmrg::fail(c, TDMRG_EINVAL, "alloc_count: null argument");
    *count = c->alloc_calls;
    *bytes = c->alloc_bytes;
    return TDMRG_OK;
}

int tdmrg_hpsi_tensor_flops(tdmrg_ctx* c, int a, int b, double* flops) {
    if (!c || !flops) return tdmrg::fail(c, TDMRG_EINVAL, "hpsi_tensor_flops: null argument");
    if (!c->ham_set) return tdmrg::fail(c, TDMRG_ESTATE, "hpsi_tensor_flops: Hamiltonian not set");
    tdmrg::Plan* p = nullptr;
    int rc = tdmrg::get_ham_plan(c, a, b, &p);
    if (rc) return rc;
    double f = 0.0;
    if (p->oz.ready) {
        const int S = p->oz.S;
        const double groups = S * (S + 1) / 2;
        for (const tdmrg::OzStage& st : p->oz.st)
            for (const tdmrg::OzTile& t : st.tiles) {
                const tdmrg::OzTask& k = st.tasks[t.task];
                if (S <= 4) {
                    // persistent kernel: per 64-wide K chunk and 16-wide k-step, A slice s times the
                    // B slices 1..S+1-s in one MMA of M = 64, N = (S + 1 - s) 64
                    f += (double)k.kchunks * 4 * groups * 2.0 * 64 * 64 * 16;
                } else {
                    // per 64-wide K chunk: 4 k-steps x S(S+1)/2 MMAs of 128 x 2n_t x 16
                    const int nval = k.N - t.n0 < 32 ? k.N - t.n0 : 32;
                    const int n_t = (nval + 7) & ~7;
                    f += (double)k.kchunks * 4 * groups * 2.0 * 128 * (2 * n_t) * 16;
                }
            }
    }
    *flops = f;
    return TDMRG_OK;
}

int tdmrg_hpsi_thin_flops(tdmrg_ctx* c, int a, int b, double* flops) {
    if (!c || !flops) return tdmrg::fail(c, TDMRG_EINVAL, "hpsi_thin_flops: null argument");
    if (!c->ham_set) return tdmrg::fail(c, TDMRG_ESTATE, "hpsi_thin_flops: Hamiltonian not set");
    tdmrg::Plan* p = nullptr;
    int rc = tdmrg::get_ham_plan(c, a, b, &p);
    if (rc) return rc;
    *flops = p->oz.ready ? p->oz.st[0].thin_flops + p->oz.st[1].thin_flops : 0.0;
    return TDMRG_OK;
}

int tdmrg_fp64_peak(int device, double* dmma, double* dfma) {
    if (!dmma || !dfma) return tdmrg::fail(nullptr, TDMRG_EINVAL, "fp64_peak: null output");
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return tdmrg::fail(nullptr, TDMRG_ECUDA, "fp64_peak: bad device"); }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * 4, threads = 256;
    double* buf = nullptr;
    cudaEvent_t e0, e1;
    int rc = TDMRG_OK;
    if (cudaMalloc(&buf, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaSetDevice(prev);
        return tdmrg::fail(nullptr, TDMRG_ENOMEM, "fp64_peak: allocation");
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    k_dmma_peak<<<blocks, threads>>>(buf, 0.5);   // warm-up
    cudaEventRecord(e0);
    k_dmma_peak<<<blocks, threads>>>(buf, 0.25);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    // one m8n8k4 MMA per warp = 8*8*4 multiply-adds = 512 flops; 4 per iteration
    *dmma = 512.0 * 4 * kIters * ((double)blocks * threads / 32) / (ms * 1e-3) / 1e12;
    k_dfma_peak<<<blocks, threads>>>(buf, 1.0000001, 1e-9);
    cudaEventRecord(e0);
    k_dfma_peak<<<blocks, threads>>>(buf, 1.0000001, 1e-9);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *dfma = 2.0 * 8 * kIters * ((double)blocks * threads) / (ms * 1e-3) / 1e12;
    if (cudaGetLastError() != cudaSuccess) rc = tdmrg::fail(nullptr, TDMRG_ECUDA, "fp64_peak: kernel failed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaSetDevice(prev);
    return rc;
}

}  // extern "C"
