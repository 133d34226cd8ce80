/*
 * tdmrg.h -- C ABI of the GB300 hot path of time-step-targeting DMRG with
 * Krylov time evolution (Alvarez, Dias da Silva, Ponce, Dagotto,
 * arXiv:1103.5391).
 *
 * The library holds one superblock L u R (Sec. II.B): the sector tables of the
 * left and right blocks, block operators split into sector blocks, and the
 * Hamiltonian as block terms plus connections across the left/right boundary
 * (Sec. IV, "Hamiltonian connections").  On that superblock it applies H psi,
 * applies local excitation operators (Eq. b), advances a targeted state by
 * Krylov time evolution (Sec. II.A Eq. lanczosevolution, Sec. II.C
 * Eq. lanczosevolution2), forms the weighted reduced density matrix of the
 * targets (Eq. rdensitymatrix with the weights of Sec. II.C) and its
 * eigendecomposition, and measures expectation values (Eq. generalcorrelation
 * with one local operator per block).
 *
 * Conventions used by every call
 *   - Complex numbers are tdmrg_c64 = {re, im} doubles, the layout of
 *     cuDoubleComplex and torch.complex128.
 *   - A quantum number is a pair (n_up, n_dn).  Sector tables must be given in
 *     strictly ascending lexicographic order of (n_up, n_dn).
 *   - The wave function of superblock sector Q = (N_up, N_dn) is the
 *     concatenation, over left sectors q in table order whose partner
 *     r = Q - q exists on the right, of the blocks Psi_q of shape
 *     dL(q) x dR(r), row-major (left index slow).  tdmrg_sector_size gives
 *     its length.
 *   - Superblock basis |alpha>|beta> = (left creation string)(right creation
 *     string)|0>.  A term "coeff * A_L B_R" is the fermionic product with the
 *     left operator written first; the library applies it as
 *     coeff * (A P_L) (x) B when B is fermion-odd, P_L = (-1)^{N_L}, and as
 *     coeff * A (x) B otherwise.  On a sector block:
 *       Psi'_{q_out} += coeff * s(q_in) * A[q_out<-q_in] Psi_{q_in} B[r_out<-r_in]^T.
 *   - Pointers named *_d are device pointers on the context's device; all
 *     other pointers are host pointers.  Device work is enqueued on the
 *     context's stream and is asynchronous unless a call says it synchronises.
 *     The caller owns every buffer it passes; the library owns copies of the
 *     operators and its workspace.
 *   - Every call returns TDMRG_OK (0) or a negative error code and never
 *     aborts; tdmrg_last_error(ctx) describes the last failure on that ctx.
 *   - A context is not thread-safe: use one context per host thread.
 */
#ifndef TDMRG_H
#define TDMRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdmrg_ctx tdmrg_ctx;
typedef struct { double re, im; } tdmrg_c64;

enum tdmrg_status {
    TDMRG_OK = 0,
    TDMRG_EINVAL = -1,     /* bad argument (null pointer, size, unknown op id)            */
    TDMRG_ENOMEM = -2,     /* device allocation failed or the HBM budget would be exceeded */
    TDMRG_ESECTOR = -3,    /* inconsistent quantum numbers (unknown sector, bad block dims) */
    TDMRG_ECUDA = -4,      /* a CUDA runtime call failed                                    */
    TDMRG_ETIMEOUT = -5,   /* a bounded device wait ran out                                 */
    TDMRG_ESTATE = -6      /* call out of order (e.g. apply_h before set_hamiltonian)       */
};

enum tdmrg_side { TDMRG_LEFT = 0, TDMRG_RIGHT = 1 };

/* Arithmetic of the superblock products (H psi, excitations, expectation values).
 * Lanczos orthogonalisation, norms, the tridiagonal exponential and rho_L always run in FP64. */
enum tdmrg_prec {
    TDMRG_FP64 = 0,        /* complex FP64 products (DMMA tensor-core path)                          */
    TDMRG_OZAKI_BF16 = 1   /* FP64 operands split into bf16 slices, exact FP32 tensor-core products,
                              FP64 recombination; accuracy set by ozaki_slices                       */
};

typedef struct {
    int device;            /* CUDA device ordinal                                         */
    void* stream;          /* cudaStream_t to enqueue on; NULL = legacy default stream     */
    int prec;              /* enum tdmrg_prec                                               */
    int ozaki_slices;      /* bf16 slices per operand for TDMRG_OZAKI_BF16 (2..7)           */
    int nk_max;            /* largest Krylov dimension n_K accepted by tdmrg_evolve (<=32)  */
    double breakdown_tol;  /* Lanczos stops when beta_{j+1} <= tol * max(1, |alpha_j|)      */
    size_t hbm_budget;     /* bytes the context may allocate on the device; 0 = unlimited   */
} tdmrg_opts;

/* Fill *o with defaults: device 0, default stream, FP64, 4 slices, nk_max 16, tol 1e-12, no budget. */
void tdmrg_default_opts(tdmrg_opts* o);

/* Create a context on o->device.  *out receives an opaque handle owned by the library. */
int tdmrg_create(tdmrg_ctx** out, const tdmrg_opts* o);
/* Release the context and all device memory it owns (synchronises its stream). */
int tdmrg_destroy(tdmrg_ctx* ctx);
/* Change the stream later calls enqueue on (e.g. torch.cuda.current_stream().cuda_stream). */
int tdmrg_set_stream(tdmrg_ctx* ctx, void* stream);
/* Change the arithmetic of superblock products (enum tdmrg_prec) and the number of Ozaki slices. */
int tdmrg_set_precision(tdmrg_ctx* ctx, int prec, int ozaki_slices);
/* Text of the last error on ctx (a static string when ctx is NULL). */
const char* tdmrg_last_error(tdmrg_ctx* ctx);

/* Block basis of one side (Sec. II.B: alpha in L, beta in R).  nsec sectors, qn[2*s] = n_up,
 * qn[2*s+1] = n_dn in strictly ascending lexicographic order, dim[s] >= 1.
 * Setting a block drops every operator, Hamiltonian and plan of that side.
 * Errors: EINVAL (nsec < 1, null), ESECTOR (order, dims). */
int tdmrg_set_block(tdmrg_ctx* ctx, int side, int nsec, const int32_t* qn, const int32_t* dim);

/* Block operator op_id (>= 0) on one side, given as nblk dense sector blocks.
 * blk_qn[4*b..4*b+3] = (out n_up, out n_dn, in n_up, in n_dn); the data of all blocks is
 * concatenated in that order, block b being dim(out) x dim(in) row-major.  fermion_odd = 1 marks an
 * operator that changes the particle number parity (c, c^dag); for a right operator it makes the
 * library apply the left parity P_L (Sec. II.B: reordering fermions costs at most a sign).
 * data may be a host (data_on_device = 0) or device pointer; the library copies it.
 * Redefining an op_id replaces it and invalidates plans that use it.
 * Errors: EINVAL, ESECTOR (unknown sector), ENOMEM. */
int tdmrg_set_op(tdmrg_ctx* ctx, int side, int op_id, int fermion_odd, int nblk, const int32_t* blk_qn,
                 const tdmrg_c64* data, int data_on_device);

/* H = H_L (x) 1 + 1 (x) H_R + sum_k coeff[k] * opL[k] opR[k]  (Sec. IV; Hubbard H of Sec. III.B).
 * opHL is a left op id, opHR a right op id (-1 = absent); opL[k] / opR[k] are left / right op ids of
 * connection k, coeff[k] its complex amplitude.  The caller includes both Hermitian halves
 * (e.g. -t c^dag_i c_j and +t c_i c^dag_j).  Errors: EINVAL, ESTATE (blocks not set). */
int tdmrg_set_hamiltonian(tdmrg_ctx* ctx, int opHL, int opHR, int nconn, const int32_t* opL,
                          const int32_t* opR, const tdmrg_c64* coeff);

/* Time-dependent Hamiltonian inside a captured step (the time-dependent Hamiltonians of Sec. I, e.g. a
 * quench or a Peierls-phased pulse on the boundary hopping): coeff_d is a device array of nconn
 * tdmrg_c64 values, the coefficients of the connections in the order given to tdmrg_set_hamiltonian.
 * From this call on, every superblock product of the Hamiltonian reads connection k's coefficient from
 * coeff_d[k] when it runs, instead of the value given to tdmrg_set_hamiltonian, so the caller may change
 * the array between steps (a copy or a kernel on the stream, also as nodes of a captured CUDA graph)
 * without any rebuild; H_L and H_R keep coefficient 1.  The caller keeps the array valid while it is
 * set; NULL returns to the static coefficients; tdmrg_set_hamiltonian also clears it.  Plans are
 * rebuilt on their next use (the call synchronises the stream).  With values equal to the static
 * coefficients the FP64 path gives the same bits; the tensor path then folds the coefficients into the
 * per-product slices of the intermediates instead of the operator slices, equal within its slicing
 * error.  Errors: ESTATE (no Hamiltonian). */
int tdmrg_set_coefficients(tdmrg_ctx* ctx, const tdmrg_c64* coeff_d);

/* Length of the sector-Q wave function (number of complex entries; 0 if Q has no pairs). */
int tdmrg_sector_size(tdmrg_ctx* ctx, int n_up, int n_dn, int64_t* dim_out);

/* out_d = H psi_d in sector Q (Sec. IV).  Both are device vectors of tdmrg_sector_size entries and
 * must not overlap.  Errors: EINVAL, ESTATE, ENOMEM, ECUDA. */
int tdmrg_apply_h(tdmrg_ctx* ctx, int n_up, int n_dn, const tdmrg_c64* psi_d, tdmrg_c64* out_d);

/* Excitation out_d = (opL P_L^{odd(opR)}) (x) opR  psi_d from sector Q_in to Q_out (Eq. b with a
 * local operator on each block; -1 = identity on that block, not both).  Errors as apply_h. */
int tdmrg_apply_op(tdmrg_ctx* ctx, int opL, int opR, int n_up, int n_dn, const tdmrg_c64* psi_d,
                   int n_up_out, int n_dn_out, tdmrg_c64* out_d);

/* Krylov advance (Sec. II.A-II.C).  From phi(t) = phi_d in sector Q, builds nk Lanczos vectors
 * started at phi (full re-orthogonalisation, two classical Gram-Schmidt passes, FP64), diagonalises
 * T = S^dag D S and writes targets_d[x] = ||phi|| V^dag S^dag e^{-i D t_x} S e_0 ~ e^{-i H t_x} phi
 * for x = 0..n_v-1 (t_x host array, t_x >= 0).  targets_d is a host array of n_v device pointers,
 * each a sector-Q vector; a target may alias phi_d (phi is copied into the Krylov workspace before
 * any target is written), targets must not alias each other.
 * Lanczos stops early at breakdown; tdmrg_evolve_info reports the dimension used and the error
 * estimate.  nk in 1..nk_max.  Errors: EINVAL, ESTATE, ENOMEM, ECUDA. */
int tdmrg_evolve(tdmrg_ctx* ctx, int n_up, int n_dn, const tdmrg_c64* phi_d, int n_v, const double* t_x,
                 int nk, tdmrg_c64* const* targets_d);

/* Ground state in sector Q (the ground-state targeting of Sec. II.B, needed at every DMRG step):
 * `restarts` times, nk Lanczos steps started at psi_d (full re-orthogonalisation, FP64), the lowest
 * eigenvector of the tridiagonal (bisection on its Sturm count, then inverse iteration, FP64) combined
 * in place into psi_d, normalised.  psi_d (device, sector Q) is the start vector on entry and the ground
 * state on return; *energy (host, nullable) receives the lowest Ritz value of the last restart.  The
 * call synchronises the stream once at the end.  Errors: EINVAL (nk outside 2..nk_max, restarts < 1),
 * ESTATE, ENOMEM, ECUDA, ETIMEOUT. */
int tdmrg_ground_state(tdmrg_ctx* ctx, int n_up, int n_dn, tdmrg_c64* psi_d, int nk, int restarts, double* energy);

/* Batching of independent problems (several superblocks, e.g. the time evolutions of different jobs):
 * tdmrg_direct_sum loads into ctx the direct sum of the superblocks of nsrc source contexts, each with
 * its sector Q_k = (Q[2k], Q[2k+1]) (host): the sectors of source k are shifted apart (left n_up by
 * 4096 k, the right sectors so that Q_k lands on the common sector Qsum = (4096 nsrc, 4096)), so no
 * product of the sum pairs blocks of different sources, and source k's operator id becomes 2^20 k + id.
 * The vector of ctx in Qsum is the concatenation of the sources' vectors in their sectors Q_k, in source
 * order: seg_off (host, nsrc + 1, nullable) receives their offsets, Qsum (host, 2, nullable) the common
 * sector.  One H psi of ctx is then one grouped product over all sources (Sec. IV).  Sources keep their
 * own data (ctx holds copies); their quantum numbers must lie in 0..2047 and their coefficients be
 * static.  Synchronises the streams.  Errors: EINVAL, ESTATE (a source without Hamiltonian), ESECTOR,
 * ENOMEM, ECUDA. */
int tdmrg_direct_sum(tdmrg_ctx* ctx, int nsrc, tdmrg_ctx* const* src, const int32_t* Q, int32_t* Qsum, int64_t* seg_off);

/* tdmrg_evolve for nseg independent problems side by side in one vector of sector Q (e.g. a direct sum):
 * segment s is elements [off_s, off_s + seg_len[s]) (host lengths, adding up to the sector size); each
 * segment gets its own Lanczos recursion (norm, alpha, beta, breakdown, re-orthogonalisation), its own
 * tridiagonal exponential and targets, exactly as tdmrg_evolve would give it alone up to the order of
 * the FP64 reductions, while every H psi is one product over all segments.  targets_d[x] are full-length
 * vectors (segment s of target x is the evolution of segment s of phi_d).  nseg is at most the number of
 * co-resident blocks of the orthogonalisation (one per SM).  Errors: as tdmrg_evolve. */
int tdmrg_evolve_segments(tdmrg_ctx* ctx, int n_up, int n_dn, const tdmrg_c64* phi_d, int nseg, const int64_t* seg_len,
                          int n_v, const double* t_x, int nk, tdmrg_c64* const* targets_d);
/* Per segment of the last tdmrg_evolve_segments with these (Q, nk, nseg): Krylov vectors used and the
 * error estimate (host arrays of nseg, nullable).  Synchronises.  Errors: ESTATE, ECUDA, ETIMEOUT. */
int tdmrg_evolve_segments_info(tdmrg_ctx* ctx, int n_up, int n_dn, int nk, int nseg, int* nk_used, double* err);

/* Results of the last tdmrg_evolve: Krylov dimension used, a-posteriori error estimate
 * ||phi|| beta_n |[e^{-i T t_{n_v-1}}]_{n-1,0}| (Saad), and optionally alpha[0..n-1], beta[0..n-1]
 * (beta[j] couples v_j and v_{j+1}; beta[n-1] is the residual).  Synchronises the stream. */
int tdmrg_evolve_info(tdmrg_ctx* ctx, int* nk_used, double* err_est, double* alpha, double* beta);

/* Weights of time-step targeting (Sec. II.C): n = n_v + 1 states including the ground state,
 * Omega = 1/(n+3); 2 Omega for the ground state, the first and the last time target, Omega for the
 * others.  w_gs (host) gets the ground-state weight, w (host, n_v) the target weights.  n_v >= 2. */
int tdmrg_tst_weights(int n_v, double* w_gs, double* w);

/* Number of complex entries of rho_L (sum over left sectors of dL^2) and of eigenvalues (sum dL). */
int tdmrg_rho_size(tdmrg_ctx* ctx, int64_t* rho_entries, int64_t* n_evals);

/* Weighted reduced density matrix (Eq. rdensitymatrix):
 *   rho_L(q) = sum_l w[l] Psi_l(q) Psi_l(q)^dag / <psi_l|psi_l>
 * over ntargets (1..12) states psi_d[l] (host array of device pointers) in sectors Q[2l], Q[2l+1] (host).
 * rho_d receives every left sector's dL x dL block, row-major, packed in left-table order (zero for
 * sectors no target reaches).  Errors: EINVAL, ESTATE, ENOMEM, ECUDA. */
int tdmrg_density_matrix(tdmrg_ctx* ctx, int ntargets, const int32_t* Q, const tdmrg_c64* const* psi_d,
                         const double* w, tdmrg_c64* rho_d);

/* Real-basis variant of time-step targeting (on = 1; 0 = off, the default): tdmrg_density_matrix then
 * forms Re rho_L = sum_l w_l (Re Psi_l(q) Re Psi_l(q)^T + Im Psi_l(q) Im Psi_l(q)^T) / <psi_l|psi_l>,
 * i.e. the real and imaginary parts of every target targeted apart with its weight (Eq. rdensitymatrix
 * on real states; the paper is silent on complex targets).  Re rho_L is real symmetric, so its
 * eigenvectors from tdmrg_rho_eig are real and block operators renormalised with them stay real; the
 * library detects real operators (zero imaginary parts, tdmrg_set_op) and skips their imaginary
 * products, half the work of a complex product.  Errors: EINVAL (null context). */
int tdmrg_set_real_basis(tdmrg_ctx* ctx, int on);

/* The same for either block (side 0: rho_L as above; side 1: the right block's matrix, needed when a
 * sweep moves left, rho_R(r) = sum_l w[l] sum_{q: Q_l - q = r} Psi_l(q)^T conj(Psi_l(q)) / <psi_l|psi_l>,
 * i.e. rho_R[b, b'] = sum_a Psi[a, b] conj(Psi[a, b']), packed per right sector).  tdmrg_rho_size_side
 * gives its sizes.  Errors as above, EINVAL for a side other than 0 or 1. */
int tdmrg_density_matrix_side(tdmrg_ctx* ctx, int side, int ntargets, const int32_t* Q,
                              const tdmrg_c64* const* psi_d, const double* w, tdmrg_c64* rho_d);
int tdmrg_rho_size_side(tdmrg_ctx* ctx, int side, int64_t* rho_entries, int64_t* n_evals);

/* Eigendecomposition of a packed rho_L (as written by tdmrg_density_matrix) to FP64 accuracy per sector
 * (dL <= 512): FP32 Jacobi seed, FP64 iterative refinement (Ogita-Aishima) with re-seeding of coupled
 * clusters.
 * evals_d (sum dL doubles) gets each sector's eigenvalues in descending order; evecs_d (packed like
 * rho) gets U with rho(q) = U diag(evals) U^dag, column k of U the k-th eigenvector.  This feeds the
 * truncation of Sec. II.B.  Errors: EINVAL, ESTATE, ECUDA. */
int tdmrg_rho_eig(tdmrg_ctx* ctx, const tdmrg_c64* rho_d, double* evals_d, tdmrg_c64* evecs_d);

/* tdmrg_rho_eig for the matrix of either block (packed over that side's sectors). */
int tdmrg_rho_eig_side(tdmrg_ctx* ctx, int side, const tdmrg_c64* rho_d, double* evals_d, tdmrg_c64* evecs_d);

/* tdmrg_density_matrix_side followed by tdmrg_rho_eig_side in one call, with the same results (Eq.
 * rdensitymatrix, then the truncation input of Sec. II.B): when the eigensolver runs its sectors in two
 * groups (the sectors with the longest Jacobi seeds on a second stream), the rho blocks of that group are
 * formed on its stream too, so that its seeds start before the other sectors' blocks are done.
 * Arguments as the two calls; rho_d is written and then decomposed.  Errors as the two calls. */
int tdmrg_density_eig(tdmrg_ctx* ctx, int side, int ntargets, const int32_t* Q, const tdmrg_c64* const* psi_d,
                      const double* w, tdmrg_c64* rho_d, double* evals_d, tdmrg_c64* evecs_d);

/* Truncation of the left block to at most m states (Sec. I: a block keeps the m most probable states of
 * its reduced density matrix).  evals_d: rho_L's eigenvalues in the packed layout of tdmrg_rho_eig (per
 * left sector, descending).  Kept set: the m largest eigenvalues over all sectors; eigenvalues within
 * 1e-12 lambda_max of the m-th largest are ties, broken by (sector index, eigen index) ascending, so
 * every sector keeps its leading eigenvectors.  kept_d (device, one int per left sector) receives the
 * states kept per sector (all of them when the block has at most m); discarded_d (device, one double,
 * nullable) the sum of the dropped eigenvalues (the truncation error).  Synchronises the stream once to
 * upload the sector tables.  Errors: EINVAL (m < 1, more than 1024 sectors), ESTATE, ECUDA. */
int tdmrg_truncate(tdmrg_ctx* ctx, const double* evals_d, int m, int32_t* kept_d, double* discarded_d);

/* tdmrg_truncate for either block (evals_d and kept_d over that side's sectors). */
int tdmrg_truncate_side(tdmrg_ctx* ctx, int side, const double* evals_d, int m, int32_t* kept_d, double* discarded_d);

/* Operator of one side renormalised into the kept basis (Sec. I): O' = U^dag O U sector block by sector
 * block, O'[q_out <- q_in] = U(q_out)[:, :k(q_out)]^dag O[q_out <- q_in] U(q_in)[:, :k(q_in)].
 * U_d: per sector of that side a dim x dim row-major matrix whose column k is the k-th eigenvector
 * (the layout of tdmrg_rho_eig); kept (host, one int per sector of that side) the kept counts k(q).
 * out_d (device) receives, for every block of the operator in the order it was set whose two kept
 * counts are nonzero, the k(q_out) x k(q_in) block row-major, concatenated; *nblk_out (host, nullable)
 * their number.  FP64 grouped products; allocates a scratch buffer and synchronises the stream.
 * Errors: EINVAL (unknown op id, kept count outside 0..dim), ESTATE, ENOMEM, ECUDA. */
int tdmrg_renormalize_op(tdmrg_ctx* ctx, int side, int op_id, const tdmrg_c64* U_d, const int32_t* kept,
                         tdmrg_c64* out_d, int* nblk_out);

/* A block operator given as sector blocks: nblk blocks, blk_qn[4*b..4*b+3] = (out n_up, out n_dn, in n_up,
 * in n_dn), data_d (device) the blocks row-major, concatenated in that order (the layout of tdmrg_set_op). */
typedef struct {
    int nblk;
    const int32_t* blk_qn;
    const tdmrg_c64* data_d;
} tdmrg_blocks;

/* Sector table of the block K enlarged by one Hubbard site (Sec. I: blocks grow by one site per step;
 * Sec. II.B: the superblock is (block + site) + (site + block)).  side 0: K + site (K's sites first),
 * side 1: site + K.  K: nsec sectors qn[2s], qn[2s+1] ascending, dims dim[s] >= 1 (host).  Writes (host,
 * each nullable) the number of enlarged sectors, their quantum numbers and dimensions (capacity cap
 * sectors), the number of blocks of the new edge operators c^dag'_up, c^dag'_dn, and the complex entries of
 * the three outputs of tdmrg_enlarge (H', c^dag'_up, c^dag'_dn).  No device work.
 * Errors: EINVAL (side, capacity), ESECTOR (table not ascending, dim < 1). */
int tdmrg_enlarge_size(int side, int nsec, const int32_t* qn, const int32_t* dim, int cap, int* nsec_out,
                       int32_t* qn_out, int32_t* dim_out, int32_t* nblk_cdag, int64_t* entries);

/* Operators of the enlarged block (Hubbard site: U n_up n_dn, bond -t to K's edge site):
 *   side 0 (K + site): H' = H_K x 1 + 1 x U n_up n_dn - t sum_s [(c^dag_K,s P_K) x c_s + (P_K c_K,s) x c^dag_s],
 *                      c^dag'_s = P_K x c^dag_s;
 *   side 1 (site + K): H' = U n_up n_dn x 1 + 1 x H_K - t sum_s [(c^dag_s P) x c_K,s + (P c_s) x c^dag_K,s],
 *                      c^dag'_s = c^dag_s x 1,
 * with P_K, P the parities of K and of the site, the site states |0>, |dn>, |up>, |up dn> created as
 * c^dag_up c^dag_dn |0>, and the enlarged basis the Kronecker basis sorted stably by quantum number (the
 * table of tdmrg_enlarge_size).  H (H_K, sector-diagonal blocks) and cdag[2] (K's edge c^dag_up, c^dag_dn)
 * are device blocks of K.  H_out (device) receives every enlarged sector's dim x dim block in table order;
 * cdag_out[s] (device) the blocks of c^dag'_s, one per enlarged sector Q that it maps out of, in table
 * order of Q, each dim(Q + e_s) x dim(Q); cdag_qn_out[s] (host, 4 ints per block, nullable) their quantum
 * numbers in tdmrg_set_op's layout; n_out[s] (device, nullable, each nullable) the density n_s of the new
 * site (1 x n_s or n_s x 1), laid out like H_out.  One placement launch into the zeroed outputs;
 * synchronises the stream.
 * Errors: EINVAL, ESECTOR (a block of H off the diagonal, a c^dag block that does not raise n_s by one),
 * ENOMEM, ECUDA. */
int tdmrg_enlarge(tdmrg_ctx* ctx, int side, int nsec, const int32_t* qn, const int32_t* dim, const tdmrg_blocks* H,
                  const tdmrg_blocks* cdag, double t, double U, tdmrg_c64* H_out, tdmrg_c64* const* cdag_out,
                  int32_t* const* cdag_qn_out, tdmrg_c64* const* n_out);

/* Enlargement on the two-leg ladder (Sec. III.A Fig. 2: 8 x 2 ladder; Sec. III.B: 2 x 4 ladders), where a
 * new site bonds to two sites of K: as tdmrg_enlarge, with nedge (1 or 2) bonds of the new site, to K's edge
 * site (c^dag in cdag[0], cdag[1], hopping t[0]) and to the second site from the edge (cdag[2], cdag[3],
 * t[1]); a zero t[e] leaves that bond out (cdag[2e], cdag[2e+1] must still be valid block lists, possibly
 * empty).  With carry_out (device, nullable; each entry non-null) K's edge is carried into the enlarged
 * block as its second site from the edge: carry_out[s] receives c^dag_{K edge, s} x 1 (side 0) or
 * P x c^dag_{K edge, s} (side 1, P the site parity) with the block list and layout of cdag_out[s]
 * (tdmrg_enlarge_size's entries[1 + s]).  nedge = 1 without carry_out is tdmrg_enlarge.  The second
 * bond's terms fall on the sub-blocks of the first's and are added by a second placement launch, the
 * carried edge by a third; synchronises the stream.
 * Errors: as tdmrg_enlarge; EINVAL also for nedge outside 1..2, t NULL or a NULL carry_out entry. */
int tdmrg_enlarge_bonds(tdmrg_ctx* ctx, int side, int nsec, const int32_t* qn, const int32_t* dim,
                        const tdmrg_blocks* H, int nedge, const tdmrg_blocks* cdag, const double* t, double U,
                        tdmrg_c64* H_out, tdmrg_c64* const* cdag_out, int32_t* const* cdag_qn_out,
                        tdmrg_c64* const* n_out, tdmrg_c64* const* carry_out);

/* Operator op_id of one side defined as the adjoint of operator src_id of the same side (block (q_in, q_out)
 * = the conjugate transpose of block (q_out, q_in); same fermion parity): e.g. c from c^dag for the
 * Hamiltonian's boundary terms.  Synchronises the stream.  Errors: EINVAL (unknown src_id, op_id < 0 or equal
 * to src_id), ENOMEM, ECUDA. */
int tdmrg_set_op_adjoint(tdmrg_ctx* ctx, int side, int op_id, int src_id);

/* Wave-function transformation of a target (Sec. II.B: transporting the targets from one superblock to
 * the next during a finite sweep).  Block bases are Kronecker products sorted stably by quantum number:
 * a sector of an enlarged left block K + site runs over K's sectors in order, a sector of an enlarged
 * right block site + K over the site states (0,0), (0,1), (1,0), (1,1) in order, each followed by the
 * states of K's matching sector.  U_d and V_d are in the layout of tdmrg_rho_eig: per sector of the
 * block they belong to, in table order, a dim x dim row-major matrix whose first columns are the kept
 * states (kept[s], kept_next[s] of them; host arrays, one count per sector).
 *
 * tdmrg_wft_right, the centre moves one site to the right: `from` holds (L_enl, R_enl) with
 * R_enl = site + R_b, `to` holds (L_enl', R_enl') with L_enl' = K + site.  U_d: rho_L's eigenvectors of
 * `from`'s left block, kept the kept counts there (K); V_d: over `to`'s right block R_enl', whose first
 * kept_next columns per sector are R_b (the truncation that made R_b).  Psi' = (U^dag Psi) re-indexed,
 * with R_b's states expanded in R_enl'.
 * tdmrg_wft_left, the centre moves one site to the left: `from` holds (L_enl = L_b + site, R_enl), `to`
 * holds (L_enl', R_enl' = site + K).  U_d: rho_R's eigenvectors of `from`'s right block (tdmrg_rho_eig_side
 * with side 1), kept there (K); V_d: over `to`'s left block L_enl', whose first kept_next columns per
 * sector are L_b.  Psi' = (Psi conj(U)) re-indexed, with L_b's states expanded in L_enl'.
 *
 * psi_d: the target in `from`'s sector Q = (n_up, n_dn); out_d: the result in `to`'s sector Q (cleared
 * first).  No fermion sign arises (the moved site keeps its place in the lattice order).  Two grouped FP64
 * launches on `from`'s stream; allocates scratch and synchronises.  Errors: EINVAL (null, kept counts
 * outside 0..dim), ESTATE, ESECTOR (the block tables do not match the move), ENOMEM, ECUDA. */
int tdmrg_wft_right(tdmrg_ctx* from, int n_up, int n_dn, const tdmrg_c64* psi_d, const tdmrg_c64* U_d,
                    const int32_t* kept, const tdmrg_c64* V_d, const int32_t* kept_next, tdmrg_ctx* to,
                    tdmrg_c64* out_d);
int tdmrg_wft_left(tdmrg_ctx* from, int n_up, int n_dn, const tdmrg_c64* psi_d, const tdmrg_c64* U_d,
                   const int32_t* kept, const tdmrg_c64* V_d, const int32_t* kept_next, tdmrg_ctx* to,
                   tdmrg_c64* out_d);

/* out_d[0] = <psi| opL opR |psi> / <psi|psi> for a sector-preserving product (Eq. generalcorrelation
 * with a = 1 local operator per block, Eq. nholondoublon; -1 = identity on that block).  out_d is
 * one device tdmrg_c64.  Errors as apply_op. */
int tdmrg_expect(tdmrg_ctx* ctx, int opL, int opR, int n_up, int n_dn, const tdmrg_c64* psi_d,
                 tdmrg_c64* out_d);

/* out_d[0] = <phi1| opL opR |phi2>, not normalised: the two-state form of Eq. generalcorrelation with
 * one local operator per block (-1 = identity on that block), e.g. one entry of a Green's function
 * <phi(t)| c_i c^dag_j |psi(t)> (Sec. I).  phi2_d lives in sector Q2 = (n_up2, n_dn2); opL opR (with
 * the fermion sign of tdmrg_apply_op) maps it to Q1 = (n_up1, n_dn1), the sector of phi1_d.  The
 * product uses a library-owned scratch vector and a fixed-order FP64 reduction; with both ids -1 it is
 * the plain overlap <phi1|phi2> (Q1 = Q2).  Errors as apply_op. */
int tdmrg_overlap_op(tdmrg_ctx* ctx, int opL, int opR, int n_up1, int n_dn1, const tdmrg_c64* phi1_d,
                     int n_up2, int n_dn2, const tdmrg_c64* phi2_d, tdmrg_c64* out_d);

/* Correlation grid, the two-state form of Eq. generalcorrelation with one local operator per block,
 * e.g. the Green's function G_ij(t) = <phi(t)| c_i c^dag_j |psi(t)> (Sec. I) on device-resident states:
 *   out_d[i * nR + j] = <phi1| opL[i] opR[j] |phi2>   (not normalised), i < nL, j < nR,
 * each product with the fermion sign of tdmrg_apply_op (-1 = identity on that block, not both in one
 * product); phi2_d lives in sector Q2 = (n_up2, n_dn2) and every product must map it to Q1 =
 * (n_up1, n_dn1), the sector of phi1_d.  out_d: nL * nR device tdmrg_c64.  The whole grid runs as two
 * grouped FP64 launches into library-owned scratch (nL * nR vectors of sector Q1 plus the
 * intermediates) and one fixed-order reduction per entry.  The plan and scratch are built by the first
 * call for a given (operator lists, sectors), which allocates and synchronises; later calls do neither
 * and may be captured in a CUDA graph.  Errors: EINVAL, ESTATE, ESECTOR, ENOMEM, ECUDA. */
int tdmrg_correlation(tdmrg_ctx* ctx, int nL, const int32_t* opL, int nR, const int32_t* opR, int n_up1, int n_dn1,
                      const tdmrg_c64* phi1_d, int n_up2, int n_dn2, const tdmrg_c64* phi2_d, tdmrg_c64* out_d);

/* ---- serving: continuous batching of time-evolution jobs ----------------------------------------
 * A server drives many independent time evolutions (each the repeated time step of Sec. II.C:
 * Krylov advance with n_v targets, weighted rho_L of the ground state and the targets with its
 * eigendecomposition, and observables after the step) on one GPU.  A host thread admits submitted
 * jobs in arrival order while the summed HBM footprint of the running jobs stays within the budget
 * and fewer than max_active run; every running job owns a stream, so the steps of different jobs
 * overlap on the device; a job's first step runs directly and the following steps replay a CUDA
 * graph captured from it.  Results are bit-for-bit those of the same job run alone (every kernel is
 * deterministic and a job's work never reads another job's memory), unless batching groups jobs
 * (tdmrg_server_set_batching). */
typedef struct tdmrg_server tdmrg_server;

enum tdmrg_job_status { TDMRG_JOB_QUEUED = 0, TDMRG_JOB_RUNNING = 1, TDMRG_JOB_DONE = 2, TDMRG_JOB_CANCELLED = 3,
                        TDMRG_JOB_FAILED = 4 };

typedef struct {
    tdmrg_ctx* ctx;              /* blocks, operators and H loaded; used only by the server until the job ends */
    int q_gs[2];                 /* sector of the ground state                                              */
    const tdmrg_c64* psi_gs_d;   /* ground state (device); caller-owned, must stay valid until the job ends  */
    int q[2];                    /* sector of the evolving state                                            */
    const tdmrg_c64* phi0_d;     /* initial state phi (device); copied when the job is admitted              */
    double tau;                  /* time step; targets at t_x = x tau / (n_v - 1)                           */
    int n_v, nk, steps;          /* time targets (2..11), Krylov dimension, number of time steps            */
    int nobs;                    /* observables measured after every step (0..16)                            */
    int32_t obs_opL[16], obs_opR[16];   /* left / right op ids of each observable (-1 = identity)         */
} tdmrg_job;

/* Create a server on `device`: hbm_budget bytes for the footprint of running jobs (0 = no limit),
 * at most max_active jobs at once.  Starts the server thread.  Errors: EINVAL, ECUDA. */
int tdmrg_server_create(tdmrg_server** out, int device, size_t hbm_budget, int max_active);
/* Batching of admitted jobs (one grouped launch across jobs): with max_group > 1, the queued jobs that
 * can share a time step (same precision, tau, n_v, n_K, steps and excitation sector shift, static
 * coefficients, distinct contexts, vector lengths within a factor of two) are admitted together, up to
 * max_group, and run as one group on the
 * direct sum of their superblocks (tdmrg_direct_sum): per time step one segmented Krylov advance with
 * one grouped product per Lanczos step for all members, one grouped rho_L and one eigendecomposition
 * over all members' sectors, then each member's observables.  Members finish together; a member's
 * results equal the job alone up to the order of the FP64 reductions.  A job at the front of the queue
 * without a partner waits up to window_us microseconds for one (while slots are free) before it runs
 * alone.  max_group = 1 (the default) runs every job on its own stream.  Errors: EINVAL. */
int tdmrg_server_set_batching(tdmrg_server* srv, int max_group, int window_us);
/* Groups formed so far and the jobs they ran. */
int tdmrg_server_batch_stats(tdmrg_server* srv, int* groups, int64_t* grouped_jobs);
/* Queue a job (non-blocking); *job_id identifies it.  Errors: EINVAL (bad description). */
int tdmrg_server_submit(tdmrg_server* srv, const tdmrg_job* job, int64_t* job_id);
/* Non-blocking state of a job.  obs (host, steps * nobs entries, nullable) receives the observables of
 * the finished steps in step order; step_ms (host, steps floats, nullable) the device time of each
 * finished step (CUDA events on the job's stream, queueing behind other jobs included).
 * Errors: EINVAL (unknown id). */
int tdmrg_server_poll(tdmrg_server* srv, int64_t job_id, int* status, int* steps_done, tdmrg_c64* obs, float* step_ms);
/* Stop a job after its step in flight; its slot and memory are released.  Errors: EINVAL. */
int tdmrg_server_cancel(tdmrg_server* srv, int64_t job_id);
/* Counts of queued, running and finished (done, cancelled or failed) jobs and the bytes in use. */
int tdmrg_server_stats(tdmrg_server* srv, int* queued, int* running, int* finished, size_t* bytes_in_use);
/* Stop the server thread, wait for every stream, release all job buffers (job contexts stay the caller's). */
int tdmrg_server_destroy(tdmrg_server* srv);
/* Text of the last server-level error, or of the failure of job_id when job_id >= 0. */
const char* tdmrg_server_last_error(tdmrg_server* srv, int64_t job_id);

/* H psi that allocates no device memory during the call.  The paper has no counterpart: this exists
 * for callers that may not allocate once they run -- a real-time loop that forbids allocation after
 * initialisation, a framework whose own pool owns all device memory, a plugin limited to the buffers
 * it is handed.  out_d = H psi_d in sector Q, always computed by the FP64 grouped GEMM, whatever the
 * context's precision: on a TDMRG_FP64 context the result is bit for bit that of tdmrg_apply_h; on a
 * TDMRG_OZAKI_BF16 context it is the FP64 product, which differs from tdmrg_apply_h's tensor-core
 * result by that path's slicing error.  The scratch (stage-1 intermediates, split-K partial tiles and
 * tickets) lives in a file-scope static device array of 32 MiB that every GPU loading the library
 * holds until the process exits.
 *   - The sector must be prepared during set-up by one tdmrg_apply_h or tdmrg_hpsi_flops call for
 *     Q (those may allocate); otherwise TDMRG_ESTATE.
 *   - A sector whose scratch exceeds 32 MiB is rejected with TDMRG_ENOMEM and a message giving the
 *     bytes it needs.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *     that device current; make that first call before any stream capture.
 *   - All calls share the one array, which keeps the previous call's contents (the tickets are
 *     cleared on the stream at every call): calls whose work overlaps on the GPU, from any context
 *     or stream, race -- serialise them. */
int tdmrg_apply_h_static(tdmrg_ctx* ctx, int n_up, int n_dn, const tdmrg_c64* psi_d, tdmrg_c64* out_d);

#ifdef __cplusplus
}
#endif
#endif /* TDMRG_H */
