// Internal types of libtdmrg: the sector-pair task lists that every superblock product is
// compiled into, the context, and the kernel launchers of each translation unit.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/tdmrg.h"

namespace tdmrg {

typedef double2 cplx;   // {re, im}, same layout as tdmrg_c64

// Programmatic dependent launch.  Kernels are launched with the programmatic-serialisation attribute and
// every kernel of the library starts with pdl_enter(), which waits until the previous grid of the stream
// has completed and its memory is visible: the launch of a kernel overlaps the end of the previous one,
// while every global memory access still follows the previous kernel's completion.  No kernel signals
// its dependents early (measured: blocks parked in the wait beside a running kernel slow it down).
// Without the launch attribute the wait returns at once.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// <<<grid, block, smem, s>>> with the programmatic-serialisation attribute
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
#endif

// Buffer ids a segment or task refers to; the launch passes the base pointers.
enum BufId : int8_t { BUF_OPS = 0, BUF_IN = 1, BUF_SCRATCH = 2, BUF_OUT = 3, BUF_EXTRA0 = 4 };
constexpr int kMaxBufs = 16;

// op(B) of a segment: 'N' B[k][n] at b[k*ldb+n]; 'T' at b[n*ldb+k]; 'C' conj of 'T'.
enum OpB : int8_t { OPB_N = 0, OPB_T = 1, OPB_C = 2, OPB_CN = 3 };   // OPB_CN: conj of 'N', B[k][n] = conj(b[k*ldb+n])

// One contribution  scale * dscale * A[M x K] * op(B)[K x N]  to a task's output.
struct Seg {
    int64_t a_off, b_off;     // element offsets into buffers a_buf, b_buf
    int32_t lda, ldb, K;
    int8_t a_buf, b_buf, opb;
    int8_t rflags;            // bit 0: A (with the scale) real, bit 1: B real -- their imaginary products are skipped
    int8_t opa;               // op(A): 0 A[m][k] at a[m*lda+k]; 1 at a[k*lda+m] (transposed); 2 its conjugate (FP64 kernel only)
    int32_t dscale;           // index into the launch's device real scales, -1 = none
    cplx scale;               // static complex factor (1 = none)
    int32_t dcoef = -1;       // index into the launch's device complex coefficients (connection terms), -1 = none
};

// C[M x N] (row stride ldc, buffer c_buf) = (beta ? C : 0) + sum of segments [seg_begin, seg_end).
struct Task {
    int64_t c_off;
    int32_t ldc, M, N;
    int32_t seg_begin, seg_end;
    int8_t c_buf, beta;
    int8_t herm;              // C Hermitian (M == N, beta == 0): tiles below the diagonal only, mirrored
    int8_t trans;             // C stored transposed: element (m, n) at c_off + n * ldc + m
    int32_t pad2;
};

// One CTA's work: output tile (m0, n0) (element origin) of task `task`, segments [seg_lo, seg_hi).
// A tile whose task is split along K has split >= 0: part `part` of `nparts`, partial tiles at
// partials[(split_base + part) * tile area], completion ticket counters[split].
struct Tile {
    int32_t task;
    int32_t m0, n0;
    int32_t cost;             // complex MACs, for ordering
    int32_t seg_lo, seg_hi;
    int32_t split, part, nparts, split_base;
};

// A compiled group of tasks on the device.
struct TaskList {
    std::vector<Task> tasks;
    std::vector<Seg> segs;
    std::vector<Tile> tiles;
    Task* d_tasks = nullptr;
    Seg* d_segs = nullptr;
    Tile* d_tiles = nullptr;
    double flops = 0.0;       // algorithmic real flops (8 per complex MAC)
    size_t bytes = 0;         // device bytes of the arrays below
    int nsplit = 0, npartial = 0;
    cplx* d_partials = nullptr;   // split-K partial tiles
    int* d_counters = nullptr;    // split-K tickets (zero between launches)
    int ntiles_first = 0;         // rho task lists ordered by eigensolver groups: tiles of the first group
};

// ---- tensor-core (Ozaki-sliced) form of a plan's stages, ozaki.cu
struct OzTask {            // one complex GEMM C (+)= A op(B), all of its segments K-concatenated
    int64_t c_off;
    int32_t ldc, M, N;
    int32_t arow0, brow0;  // first panel row of A' (rows) and B' (column pairs)
    int32_t aexp0, bexp0;  // first exponent of the rows / columns
    int32_t kchunks;       // 64-wide chunks of the real K (2 sum K)
    int8_t c_buf, beta, trans, pad1;
};
struct OzTile { int32_t task, m0, n0, cost; };
// An 8 x 8 output block of a thin sector-pair product (min(M, N) below the thin threshold), computed in
// FP64 by the thin warps of the persistent tensor kernel; task indexes the stage's FP64 thin tasks.
struct ThinItem { int32_t task, m0, n0, cost; };
struct OzSliceJob {        // slices the rows of A' (role 0) or columns of B' (role 1) of one operand
    int32_t role, nvec, seg_begin, seg_end, row0, exp0, ktot, use_scale, vec_prefix;
};
struct OzSliceArgs {
    const OzSliceJob* jobs;
    const int* vjob;       // job of each vector
    int njobs;
    const Seg* segs;
    __nv_bfloat16* panel;
    int* exps;
    int rows, kpad, S, nvec_total;
};
struct OzGemmArgs {
    const OzTask* tasks;
    const OzTile* tiles;
    const int* expA;
    const int* expB;
    int rowsA, rowsB;
    int* status;
    unsigned* sched;   // work queue of the persistent kernel: [0] next tile, [1] finished CTAs (zero between launches)
    const Task* ttasks;       // thin tasks (FP64 warps): tasks, segments, items grouped by CTA
    const Seg* tsegs;
    const ThinItem* titems;
    const int* tcta;          // items of CTA b: titems[tcta[b] .. tcta[b + 1]) (null: none)
};
struct OzStage {
    std::vector<OzTask> tasks;
    std::vector<OzTile> tiles;      // M = 64 tiles (the M of the kernel for S > 4 when that kernel runs)
    std::vector<OzTile> tiles128;   // M = 128 tiles of the persistent kernel (S <= 4)
    OzTile* d_tiles128 = nullptr;
    int tmw = 64;                   // tile M of the persistent kernel, chosen by the autotuner
    std::vector<OzSliceJob> ajobs, bjobs;
    std::vector<Seg> asegs, bsegs;
    std::vector<int> avjob, bvjob;   // job index of every vector
    int* d_avjob = nullptr;
    int* d_bvjob = nullptr;
    OzTask* d_tasks = nullptr;
    OzTile* d_tiles = nullptr;
    OzSliceJob* d_ajobs = nullptr;
    OzSliceJob* d_bjobs = nullptr;
    Seg* d_asegs = nullptr;
    Seg* d_bsegs = nullptr;
    __nv_bfloat16* panelA = nullptr;   // S slice planes of rowsA x kpad bf16
    __nv_bfloat16* panelB = nullptr;
    int* expA = nullptr;
    int* expB = nullptr;
    size_t panel_bytes_a = 0, panel_bytes_b = 0, exp_bytes_a = 0, exp_bytes_b = 0;
    int rowsA = 0, rowsB = 0, kpad = 0, ncolsB = 0;
    unsigned* d_sched = nullptr;
    int queue = 0;   // tile schedule of the persistent kernel: 0 static, 1 work queue (chosen by timing)
    int grid = 0;    // CTAs of the persistent kernel
    // thin sector-pair products on the FP64 warps of the persistent kernel
    std::vector<Task> ttasks;
    std::vector<Seg> tsegs;
    std::vector<ThinItem> titems;
    std::vector<int> tcta;
    Task* d_ttasks = nullptr;
    Seg* d_tsegs = nullptr;
    ThinItem* d_titems = nullptr;
    int* d_tcta = nullptr;
    double thin_flops = 0.0;   // algorithmic flops of the thin products (8 per complex MAC)
    CUtensorMap mapA, mapB, mapA128;
    OzSliceArgs sliceA{}, sliceB{};
    OzGemmArgs args{};
};
struct OzPlan {
    bool ready = false;
    int S = 0;
    OzStage st[2];
    int* status = nullptr;   // set by a tensor-core CTA whose bounded wait ran out
};

// A superblock product compiled for (terms, Q_in, Q_out): stage 1 right products, stage 2 left
// products (see plan.cu); with TDMRG_OZAKI_BF16 also their tensor-core form and the FP64 remainder.
struct Plan {
    int qin[2], qout[2];
    int64_t n_in = 0, n_out = 0, scratch = 0;   // complex entries
    TaskList stage1, stage2;
    double flops = 0.0;
    OzPlan oz;
    TaskList thin[2];
};

// The correlation grid <phi1| A_i B_j |phi2>: every product of the grid compiled into one pair of task
// lists (stage 1 into per-product scratch, stage 2 into per-product output vectors W_ij), then dots.
struct CorrPlan {
    TaskList s1, s2;
    int npairs = 0;
    int64_t n1 = 0, scratch = 0;
    cplx* T = nullptr;          // stage-1 intermediates of all products
    cplx* W = nullptr;          // npairs vectors of sector Q1
    double2* part = nullptr;    // dot partials, npairs x kCorrChunks
};
constexpr int kCorrChunks = 32;

struct BlockOp {
    int side = 0, odd = 0;
    int real = 0;             // every block has zero imaginary parts (the real-basis variant keeps operators real)
    // (out sector, in sector) -> element offset in the op pool; dims from the sector tables
    std::vector<std::tuple<int, int, int64_t>> blocks;
    int version = 0;
};

struct Side {
    std::vector<int> nup, ndn, dim;
    std::map<std::pair<int, int>, int> index;
    bool set = false;
    int find(int a, int b) const {
        auto it = index.find({a, b});
        return it == index.end() ? -1 : it->second;
    }
};

struct Term {           // coeff * (A P_L^{odd B}) (x) B; -1 = identity
    int opL, opR;
    cplx coeff;
    int conn = -1;      // index of a Hamiltonian connection (its coefficient may live on the device), -1 = none
};

struct KrylovWork {     // device workspace of tdmrg_evolve for one (Q, nk)
    int64_t n = 0;
    int nk = 0;
    cplx* V = nullptr;          // (nk + 1) x n Lanczos vectors
    cplx* w = nullptr;          // n
    double2* partA = nullptr;   // reduction partials
    double2* partB = nullptr;
    double* tri = nullptr;      // alpha[32], beta[32], beta0, resid, err
    int* flags = nullptr;       // n_used
    cplx* coef = nullptr;       // [x][k] Krylov coefficients
    unsigned* bar = nullptr;    // grid barrier of the fused orthogonalisation
    int orth_grid = 0;
    // segmented mode (independent problems side by side in one vector): per-segment tridiagonals, flags
    // and coefficients, and the CTA partition of the vector, in one device allocation
    int nseg = 0;
    std::vector<int64_t> seg_len;
    void* segmem = nullptr;
    size_t segmem_bytes = 0;
};

// One group of sectors of the rho eigensolver (eig.cu): its own tables, Jacobi records, refinement task
// lists and device-side iteration count, so that two groups run independently on two streams.
struct EigGroup {
    std::vector<int> sel;       // the group's sectors (indices into the side's sector list)
    int ns = 0;
    void* tables = nullptr;     // per-sector offsets (into the side's packed rho) and dims
    size_t tables_bytes = 0;
    double* fro = nullptr;      // per sector ||rho||_F, then the iteration count (int)
    int jac_smem = 0;           // dynamic shared memory of the Jacobi launch
    int* flags = nullptr;       // per sector: re-seed requested by the refinement
    float4* grec = nullptr;     // Jacobi rotation records of the sectors too large for V in shared memory
    int64_t grec_entries = 0;
    int* nrec = nullptr;        // per sector: rounds recorded by the last Jacobi launch (-1: skipped)
    int2* stats = nullptr;      // per sector: sweeps and SM cycles of the last seed Jacobi
    int nbig = 0, maxn_big = 0, replay_batch = 0, replay_smem = 0;
    void* oa = nullptr;         // work items of the element-wise refinement kernels, their partials and counters
    int noa = 0;
    TaskList tl_ax, tl_sg, tl_y;
};

// Workspace of the rho eigensolver (eig.cu), built once per block.  The sectors form one group, or two
// (the few largest, whose Jacobi seed is the longest, on a second stream, beside the others).
struct EigWork {
    bool ready = false;
    int64_t nrho = 0, nev = 0;
    int maxn = 0, ns = 0;
    cplx* buf = nullptr;        // 6 packed matrices: X, AX, Xh, S, G, E1
    double* lam = nullptr;
    float2* gwork = nullptr;    // FP32 Jacobi storage for sectors too large for shared memory
    int ngroups = 0;
    EigGroup grp[2];
    cudaStream_t side = nullptr;            // stream of the first group when there are two
    cudaEvent_t fork = nullptr, join = nullptr;
};

// Launch of a grouped complex GEMM (gemm_f64.cu / gemm_ozaki.cu).
struct GemmArgs {
    const Task* tasks;
    const Seg* segs;
    const Tile* tiles;
    int ntiles;
    cplx* bufs[kMaxBufs];
    const double* dscale;
    cplx* partials;
    int* counters;
    const cplx* dcoef = nullptr;   // device coefficients of the Hamiltonian connections (null: static)
};

}  // namespace tdmrg

struct tdmrg_ctx {
    tdmrg_opts opts;
    cudaStream_t stream = nullptr;
    std::string err;
    tdmrg::Side side[2];
    // op pool: one device buffer holding every operator block
    tdmrg::cplx* pool = nullptr;
    int64_t pool_cap = 0, pool_used = 0;
    std::map<int, tdmrg::BlockOp> ops[2];
    bool ham_set = false;
    std::vector<tdmrg::Term> ham;
    int ham_version = 0;
    std::map<std::tuple<int, int, int, int, int, int, int>, std::unique_ptr<tdmrg::Plan>> plans;
    std::map<std::vector<int>, std::unique_ptr<tdmrg::TaskList>> rho_plans;   // keyed by the targets' sectors
    std::map<std::vector<int>, std::unique_ptr<tdmrg::CorrPlan>> corr_plans;  // keyed by operator lists and sectors
    // generic workspace
    tdmrg::cplx* scratch = nullptr;
    int64_t scratch_cap = 0;
    std::map<std::pair<int, int>, tdmrg::KrylovWork> krylov;
    tdmrg::KrylovWork* last_krylov = nullptr;
    // reduction / misc device buffers
    double2* red = nullptr;        // partials for norms and dots
    // direct sum of superblocks (tdmrg_direct_sum): source of every left / right sector (empty otherwise),
    // and the per-(target, source) scales of the density matrix
    std::vector<int> dsum_src[2];
    int dsum_nsrc = 0;
    double* dsum_dscale = nullptr;
    size_t dsum_dscale_bytes = 0;
    struct DsumNorms { void* d = nullptr; size_t bytes = 0; int count = 0; };
    std::map<std::vector<int>, DsumNorms> dsum_norms;   // per-(target, source) ranges, keyed like rho_plans
    double* dscale = nullptr;      // device real scales (rho weights)
    tdmrg::cplx* tmp = nullptr;    // apply_op temporary for expect
    int64_t tmp_cap = 0;
    size_t allocated = 0;
    int64_t alloc_calls = 0;       // successful device allocations (cudaMalloc) made by this context
    int64_t alloc_bytes = 0;       // their total size
    int num_sms = 0;
    int64_t launches = 0;          // kernels launched by this context
    int schedule = -1;             // tile schedule of the persistent tensor kernel: -1 autotuned, 0 static, 1 queue
    int tile_m = 0;                // tile M of the persistent tensor kernel: 0 autotuned, 64, 128
    int orth_per_sm = 0;           // blocks per SM of the cooperative orthogonalisation (0: the default)
    void* trunc_tables = nullptr;  // sector tables of tdmrg_truncate
    size_t trunc_tables_bytes = 0;
    int thin_dim = 12;
    int real_basis = 0;            // tdmrg_density_matrix forms Re rho_L (targets' real and imaginary parts apart)
    const tdmrg::cplx* dcoef = nullptr;   // caller's device array of connection coefficients (null: static)             // tensor path: sector products with min(M, N) below this run on FP64 warps
    int* dstatus = nullptr;        // device word: bit 0 set when a bounded device wait ran out
    tdmrg::EigWork eig[2];         // per side (rho_L, rho_R)
};

namespace tdmrg {

// error helpers (api.cu)
struct DeviceGuard {   // makes the context's device current for the duration of a call
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int fail(tdmrg_ctx* c, int code, const std::string& msg);
int cuda_check(tdmrg_ctx* c, cudaError_t e, const char* what);
int dev_alloc(tdmrg_ctx* c, void** p, size_t bytes, const char* what);
void dev_free(tdmrg_ctx* c, void* p, size_t bytes);

// plan.cu
int build_plan(tdmrg_ctx* c, const std::vector<Term>& terms, int qin0, int qin1, int qout0, int qout1,
               Plan* out, bool to_device = true);
int64_t sector_size(const tdmrg_ctx* c, int n_up, int n_dn);
void make_tiles(TaskList& tl, int tm, int tn, int ksplit);
int upload(tdmrg_ctx* c, TaskList& tl);
void release(tdmrg_ctx* c, TaskList& tl);
int run_plan(tdmrg_ctx* c, const Plan& p, const cplx* in, cplx* out, const int* skip_flag, int skip_step);

// gemm_f64.cu: grouped complex FP64 GEMM (FP64 MMA), tile 16 x 16, split-K above kSplitK
constexpr int kTileF64 = 16;
constexpr int kSplitK = 96;
// corr: the correction mode of the eigen-refinement update, C = (I + A) B with A B in FP32
cudaError_t launch_gemm_f64(const GemmArgs& a, cudaStream_t s, const int* skip_flag, int skip_step, bool corr = false);


// api.cu: cached plan of H psi in sector (a, b), in the context's precision
int get_ham_plan(tdmrg_ctx* c, int a, int b, Plan** out);
int check_device_status(tdmrg_ctx* c);

// ozaki.cu: tensor-core superblock products
int build_oz(tdmrg_ctx* c, Plan* p, int S);
int run_oz(tdmrg_ctx* c, const Plan& p, const cplx* in, cplx* out, const int* skip_flag, int skip_step);
void release_oz(tdmrg_ctx* c, OzPlan& oz);
int oz_status(tdmrg_ctx* c, const Plan& p, int* status);

// krylov.cu
int evolve(tdmrg_ctx* c, int n_up, int n_dn, const cplx* phi, int n_v, const double* t_x, int nk,
           cplx* const* targets);
int evolve_info(tdmrg_ctx* c, int* nk_used, double* err, double* alpha, double* beta);
int ground_state(tdmrg_ctx* c, int n_up, int n_dn, cplx* psi, int nk, int restarts, double* energy);
int evolve_segments(tdmrg_ctx* c, int n_up, int n_dn, const cplx* phi, int nseg, const int64_t* seg_len, int n_v,
                    const double* t_x, int nk, cplx* const* targets);
int segments_info(tdmrg_ctx* c, int n_up, int n_dn, int nk, int nseg, int* nk_used, double* err);
cudaError_t launch_norm2(const cplx* x, int64_t n, double2* partials, int nblk, cudaStream_t s);
cudaError_t launch_dot_final(const cplx* x, const cplx* y, int64_t n, double2* partials, int nblk,
                             cplx* out, int normalise, cudaStream_t s);
constexpr int kRedBlocks = 304;   // 2 x 152 SMs: fixed, so reductions are deterministic

// density.cu
// With `grouped` (a side whose eigensolver runs two sector groups, eig_prepare done), the rho blocks of the
// first group's sectors are formed on that group's stream (forked after the target norms) and the others
// on the context stream; eig_launch(..., true) then continues each group on its stream.
int density_matrix(tdmrg_ctx* c, int side, int nt, const int32_t* Q, const cplx* const* psi, const double* w, cplx* rho,
                   bool grouped = false);
int eig_prepare(tdmrg_ctx* c, int side);
int eig_launch(tdmrg_ctx* c, int side, const cplx* rho, double* evals, cplx* evecs, bool forked);

// correlation.cu
void release_corr(tdmrg_ctx* c);

// eig.cu
int rho_eig(tdmrg_ctx* c, int side, const cplx* rho, double* evals, cplx* evecs);
void release_eig(tdmrg_ctx* c, int side);

}  // namespace tdmrg
