/*
 * nsamg -- solve phase of the GMRES + C-AMG method of arXiv:2112.14681
 * ("Neumann Series in GMRES and Algebraic Multigrid Smoothers") on one NVIDIA B300 (sm_103a).
 *
 * C ABI. Plain pointers and sizes only; no exceptions cross this boundary. Every function that
 * can fail returns an nsamg status code (0 = success, 1 = not converged, negative = error) and
 * records a message retrievable with nsamg_last_error() (thread-local).
 *
 * Memory: "host" pointers are ordinary CPU memory; "device" pointers are CUDA global memory of the
 * device that was current when the handle was created (for example torch.empty(..., device="cuda")
 * storage). All index arrays are 0-based int32 with columns sorted ascending in each row; all
 * values are float64 (IEEE binary64), vectors contiguous.
 */
#ifndef NSAMG_H
#define NSAMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------ */
#define NSAMG_OK 0                 /* converged (or a happy breakdown, beta = 0)               */
#define NSAMG_NOT_CONVERGED 1      /* maxit reached; x holds the last iterate                  */
#define NSAMG_PENDING 2            /* asynchronous request still running                       */
#define NSAMG_ERR_INVALID_ARG (-1) /* null pointer, bad size or parameter out of range         */
#define NSAMG_ERR_BAD_MATRIX (-2)  /* CSR validation failed (rowptr, column range, diagonal)   */
#define NSAMG_ERR_OOM (-3)         /* cudaMalloc failed                                        */
#define NSAMG_ERR_CUDA (-4)        /* any other CUDA runtime error (message in last_error)     */
#define NSAMG_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up                       */
#define NSAMG_ERR_NONFINITE (-6)   /* NaN/Inf met in a reduction (b, x0 or the iteration)      */
#define NSAMG_ERR_ADMISSION (-7)   /* request rejected by the admission policy                 */

/* ---- smoothers (Sec. 5.2, 5.3 and the l1-Jacobi comparison of Sec. 6.1) ------------------ */
#define NSAMG_SMOOTHER_POLY_GS 0     /* polynomial Gauss-Seidel: truncated Neumann series of (D+L)^-1 */
#define NSAMG_SMOOTHER_JACOBI_L1 1   /* x += D_l1^-1 (b - A x), d_ii = sum_j |a_ij|                  */
#define NSAMG_SMOOTHER_ILU0 2        /* ILU(0) with Neumann-series triangular solves, every level with factors */
#define NSAMG_SMOOTHER_HYBRID_ILU0 3 /* ILU(0) on the finest level, polynomial GS below (Sec. 6.2)      */

#define NSAMG_MAX_RESTART 64         /* largest supported GMRES restart length m */

/* Host CSR matrix (nrows x ncols, nnz entries). An absent matrix has nrows = 0. */
typedef struct {
  int32_t nrows, ncols;
  int64_t nnz;
  const int32_t* rowptr; /* nrows + 1 */
  const int32_t* col;    /* nnz */
  const double* val;     /* nnz */
} nsamg_csr;

/* One level of a Ruge-Stuben hierarchy built on the host (input generation).
 * A: level operator A_l. P: prolongation n_l x n_{l+1}; R = P^T: restriction n_{l+1} x n_l
 * (both absent on the coarsest level). Optional incomplete factors (ilu_L.nrows = 0 when absent):
 *   ilu_form 0, ILU(0) in row-scaled LDU form (Sec. 5.3.2): A_l ~ (I + L_s) diag(1/ilu_dinv)
 *     (I + U_s), ilu_L = L_s strictly lower, ilu_U = U_s strictly upper; ilu_dr/ilu_dc unused.
 *   ilu_form 1, ILUT with Ruiz scaling (Algorithm 2): A_l ~ (I + L_s) U, ilu_L = L_s, ilu_U = U
 *     upper with its diagonal, ilu_dr / ilu_dc the row / column scalings of U (D_r U D_c has
 *     unit row and column maxima; NULL = no scaling); ilu_dinv unused. */
typedef struct {
  nsamg_csr A, P, R, ilu_L, ilu_U;
  const double* ilu_dinv;
  int32_t ilu_form;
  const double* ilu_dr;
  const double* ilu_dc;
} nsamg_level_desc;

typedef struct {
  int32_t nlevels;
  const nsamg_level_desc* levels; /* nlevels entries, finest first */
  const double* coarse_inv;       /* dense row-major inverse of the coarsest A (n_L^2), or NULL */
} nsamg_hierarchy_desc;

/* Solve-phase parameters. Defaults from nsamg_default_params(). */
typedef struct {
  int32_t smoother;      /* NSAMG_SMOOTHER_*                                                   */
  int32_t neumann_terms; /* k terms of the polynomial GS series (k = 1 is Jacobi), >= 1          */
  int32_t ilu_terms_L;   /* terms of sum (-L_s)^j  (3 = "three Jacobi iterations", Sec. 6.2)     */
  int32_t ilu_terms_U;   /* terms of sum (-U_s)^j                                                */
  int32_t pre_sweeps;    /* sweeps before the coarse correction (forward GS direction)           */
  int32_t post_sweeps;   /* sweeps after it (backward GS direction)                              */
  int32_t coarse_sweeps; /* sweeps on the coarsest level when no dense inverse is given          */
  int32_t restart;       /* GMRES restart length m, 1..NSAMG_MAX_RESTART                         */
  int32_t vcycle_fp32;   /* 0: FP64 V-cycle. 1: FP32 matrices and vectors in the V-cycle         */
  int32_t t_exact;       /* 0: T = I - L (truncated Neumann, Algorithm 1). 1: T = (I + L)^-1    */
  int32_t use_graph;     /* 1: run each solve as one CUDA graph with device-side loop control    */
  int32_t spmv_group;    /* 0: autotune at setup (CSR with 1..32 threads per row, or a SELL-32
                            shape for matrices with >= 16384 rows); 1..32: CSR with that many
                            threads per row; -1: SELL-32 wherever available (shape sell_shape)     */
  int32_t fuse_tail;     /* 1: the V-cycle below the first level with at most 8192 rows (every
                            smoother pass with all its Neumann terms, residual, transfers and the
                            coarse solve) runs as one thread-block-cluster kernel that stages each
                            pass's source vector in shared memory; bitwise the same result as the
                            separate launches. 2: the passes below the first level with at most
                            32768 rows whose passes are all CSR row passes run as one cooperative
                            kernel over every SM (one block per SM), a bounded grid barrier
                            between dependent passes (a wait that gives up ends the solve with
                            NSAMG_ERR_TIMEOUT); bitwise the same result as the separate launches.
                            0 (default): one launch per pass. Batches ignore it.                  */
  int32_t sell_shape;    /* with spmv_group = -1: the SELL launch shape 10 K + U, K chunks of 32
                            rows per warp and U entries of each chunk staged per round: 11, 21,
                            41, 14, 18 or 22 (0 = 11). Every shape sums each row in the same order, so
                            the results do not depend on it. Ignored otherwise (the autotuner
                            picks the shape).                                                     */
  int32_t krylov_fp64;   /* 0 (default): the Gram and update kernels (Algorithm 1 steps 6 and 12)
                            form their i-dependent products in double-FP32 arithmetic (each FP64
                            value split into two FP32 parts by integer operations, TwoProduct and
                            TwoSum accumulation, Ogita-Rump-Oishi Dot2), accurate to ~2^-45 of
                            sum |a_k b_k| per product sum, because B300 issues FP64 FMAs at ~1/80
                            of its FP32 rate; vectors stay FP64 in memory, the vt . vt and vt . w
                            products and all block/grid sums stay FP64, and blocks whose data
                            leave the [2^-50, 2^60] magnitude window recompute in FP64.
                            Solves and batches keep the basis split (row-pair (hi, lo) columns).
                            1: every product and sum in FP64 (batches: an FP64 basis, products
                            in double-FP32 with a split per read).                                */
  int32_t stop_nrbe;     /* 0 (default): stop when ||b - A x|| / ||b|| <= rtol (eq. relres).
                            1: stop when the norm-wise relative backward error
                            beta(x) = ||b - A x|| / (||b|| + ||A||_inf ||x||) <= rtol (Sec. 3). Inside a
                            restart cycle the implicit residual |g_{k+1}| is tested against
                            rtol (||b|| + ||A||_inf ||x_0||) with x_0 the cycle's start (the only
                            norm of x known before the x-update); the true residual at the cycle's
                            end then decides with the exact beta(x), restarting if it fails.      */
  int32_t ranks;         /* 1 (default): smoothers couple all rows of a level. P > 1: the hybrid
                            block-Jacobi smoothing of a P-rank run (Sec. 5.2): each level's rows
                            are dealt to P contiguous blocks of ceil(n_l / P) rows, and the
                            polynomial Gauss-Seidel triangular parts keep only the couplings
                            inside a block (Jacobi across blocks); residuals use the whole level
                            operator. ILU factors are taken from the hierarchy as given (build
                            them from the block diagonal for a P-rank run). One GPU computes every
                            block; 1 <= P <= 2^20. Not with nsamg_amg_setup_solver.                */
} nsamg_params;

typedef struct {
  int32_t iters;          /* Arnoldi columns used, summed over restart cycles                   */
  int32_t restarts;       /* completed restart cycles after the first                           */
  int32_t converged;      /* 1 if ||b - A x|| / ||b|| <= rtol (with stop_nrbe: nrbe <= rtol)    */
  int32_t status;         /* same value the call returned                                       */
  double relres_true;     /* ||b - A x|| / ||b|| from the final true residual (eq. relres)      */
  double relres_implicit; /* |g_{k+1}| / ||b|| from the Givens recurrence at exit               */
  double bnorm;           /* ||b||                                                              */
  double nrbe;            /* norm-wise relative backward error ||r|| / (||b|| + ||A||_inf ||x||) of
                             the final iterate (Sec. 3)                                          */
  double orth_loss;       /* ||I - V^T V||_F of the last cycle's basis, from sqrt(2) ||L||_F (Sec. 3) */
  double sk_norm;         /* ||S_k||_2 of the last cycle, S_k = (I + U_k)^-1 U_k with U_k the strictly
                             upper part of V_k^T V_k (Sec. 3); 1 means the basis became linearly
                             dependent (see nsamg_sknorm)                                        */
} nsamg_stats;

typedef struct nsamg_handle nsamg_handle;

/* Fill *p with the defaults: POLY_GS, 2 Neumann terms, 3+3 ILU terms, 1+1 sweeps, 4 coarse
 * sweeps, m = 30, FP64 V-cycle, T = I - L, CUDA graph on, autotuned CSR kernels. */
void nsamg_default_params(nsamg_params* p);

/* Upload a host-built hierarchy (Sec. 5: A_k = R_k A_{k-1} P_k, R_k = P_k^T) and allocate the
 * GMRES workspace. The library copies everything it needs; no host pointer is kept. The split
 * A = L + D + U, D^-1 and the l1 diagonal are formed here. `cuda_stream` (a cudaStream_t, may
 * be NULL for the legacy default stream) is the stream every later call on this handle uses.
 * Errors: INVALID_ARG (null pointers, nlevels < 1, bad params), BAD_MATRIX (validation), OOM,
 * CUDA. On error *out is set to NULL. */
int nsamg_setup_hierarchy(const nsamg_hierarchy_desc* H, const nsamg_params* p, void* cuda_stream,
                          nsamg_handle** out);

/* Solve A x = b with right-preconditioned flexible one-reduce MGS-GMRES(m) whose projection
 * uses T = I - L (Algorithm 1, Sec. 4), one V-cycle per Arnoldi step (Sec. 5), restarting from
 * the true residual until ||b - A x||/||b|| <= rtol (eq. relres) or `maxit` Arnoldi steps.
 * d_b, d_x: device float64 arrays of n = A_0 rows; d_x holds x0 on entry and x on return.
 * Blocks until the solve finishes. Returns OK, NOT_CONVERGED, or an error. st may be NULL. */
int nsamg_solve(nsamg_handle* h, const double* d_b, double* d_x, double rtol, int maxit, nsamg_stats* st);

/* Same as nsamg_solve with HOST arrays: copies b and x0 to the device, solves, copies x back
 * (in stream order after the solve; on an error return h_x holds the last iterate). */
int nsamg_solve_host(nsamg_handle* h, const double* h_b, double* h_x, double rtol, int maxit, nsamg_stats* st);

/* A second solver context on the hierarchy of `parent` (a handle from nsamg_setup_hierarchy or
 * nsamg_amg_setup_solver): it shares the parent's read-only matrices, coarse inverse and tuned
 * kernel shapes and owns its own level vectors, Krylov workspace, CUDA graph and a new
 * non-blocking stream, so solves on different contexts can run at the same time from different
 * host threads (for instance one context's host copies beside another's kernels). A solve on
 * a context gives bitwise the parent's result. The parent must outlive its contexts; destroy a
 * context with nsamg_destroy. Errors: INVALID_ARG (null pointer, a batch handle, or a context as
 * parent), OOM, CUDA. On error *out is NULL. */
int nsamg_context_create(nsamg_handle* parent, nsamg_handle** out);

/* z = M^-1 r: one V-cycle with zero initial guess (Sec. 5). d_r, d_z: device float64, n entries.
 * Asynchronous on the handle's stream. */
int nsamg_apply_vcycle(nsamg_handle* h, const double* d_r, double* d_z);

/* Per-kernel entry points on a level of the handle's hierarchy (asynchronous, device arrays):
 *   nsamg_level_spmv:     y = A_l x                                     (Sec. 1, SpMV)
 *   nsamg_level_residual: r = b - A_l x                                  (eq. relres)
 *   nsamg_level_smooth:   one smoother sweep x <- x + B (b - A_l x) of the level's smoother;
 *                         backward = 1 selects the backward GS direction; x_is_zero = 1 lets the
 *                         kernels skip the A pass (x must then hold zeros or anything: it is
 *                         overwritten).
 *   nsamg_level_restrict: y_{l+1} = R_l r                                (Sec. 5)
 *   nsamg_level_prolong:  x_l += P_l e                                   (Sec. 5)
 *   nsamg_coarse_solve:   z = A_L^-1 b on the coarsest level (dense inverse, or sweeps)
 */
int nsamg_level_size(nsamg_handle* h, int level);
int nsamg_num_levels(nsamg_handle* h);
int nsamg_level_spmv(nsamg_handle* h, int level, const double* d_x, double* d_y);
int nsamg_level_residual(nsamg_handle* h, int level, const double* d_b, const double* d_x, double* d_r);
int nsamg_level_smooth(nsamg_handle* h, int level, int backward, int x_is_zero, const double* d_b, double* d_x);
int nsamg_level_restrict(nsamg_handle* h, int level, const double* d_r, double* d_y);
int nsamg_level_prolong(nsamg_handle* h, int level, const double* d_e, double* d_x);
int nsamg_coarse_solve(nsamg_handle* h, const double* d_b, double* d_z);

/* One-reduce Arnoldi kernels on caller data (Algorithm 1 steps 6-12), asynchronous on `stream`:
 *   nsamg_gram:   out[0..i] = [V_i, vt]^T vt and out[i+1..2i+1] = [V_i, vt]^T w, where V_i is the
 *                 n x i column-major block at d_V with leading dimension ldv (>= n) and vt is
 *                 column i of the same block (so the block holds i+1 columns). One pass over the
 *                 i+2 vectors, deterministic fixed-order reduction. 0 <= i < NSAMG_MAX_RESTART.
 *                 The products with V_i are formed in double-FP32 arithmetic as in a solve with
 *                 krylov_fp64 = 0 (accurate to ~2^-45 of sum |a_k b_k|); a block whose data lie
 *                 outside the [2^-50, 2^60] magnitude window is computed in FP64.
 *   nsamg_update: given beta and h[0..i] (device), writes v_i = vt / beta in place of column i
 *                 and column i+1 = w / beta - sum_{j<=i} h_j v_j; returns ||column i+1||^2 in
 *                 *d_sumsq (device). Double-FP32 products as nsamg_gram (rows outside the window
 *                 in FP64).
 *   nsamg_gram_fp64, nsamg_update_fp64: the same results with every product and sum in FP64
 *                 (the kernels of a solve with krylov_fp64 = 1).
 * All four use one library-owned device scratch per device (allocated on the first call): the
 * Gram calls share one region and counter, the update calls another. Calls of the same family
 * that overlap on the GPU (different streams, or threads without ordering) race and give wrong
 * results, so serialise them. Errors: INVALID_ARG for n <= 0, i out of range, ldv < n, null
 * pointers or beta = 0. */
int nsamg_gram(int64_t n, int i, const double* d_V, int64_t ldv, const double* d_w, double* d_out, void* stream);
int nsamg_update(int64_t n, int i, double* d_V, int64_t ldv, const double* d_w, double beta, const double* d_h,
                 double* d_sumsq, void* stream);
int nsamg_gram_fp64(int64_t n, int i, const double* d_V, int64_t ldv, const double* d_w, double* d_out, void* stream);
int nsamg_update_fp64(int64_t n, int i, double* d_V, int64_t ldv, const double* d_w, double beta, const double* d_h,
                      double* d_sumsq, void* stream);

/* The split-basis kernels a solve with krylov_fp64 = 0 runs (Algorithm 1 steps 6-12 on its own
 * basis layout), on caller data. Each entry is stored as a (hi, lo) float pair, 8 bytes per entry
 * (column j at d_Vs + 8 j lds bytes): hi = the first 24 significant bits of the FP64 value, lo
 * the next 23 (|x - hi - lo| <= 2^-46 |x|; magnitudes below 2^-103 are stored as zero). Rows are
 * stored in pairs: the 16 bytes of group g of a column are (hi_2g, hi_2g+1, lo_2g, lo_2g+1) as
 * four floats, so each column takes 8 * (n rounded up to even) bytes. When n is odd, the row-n
 * lane of the last group must be zero (nsamg_split_basis and nsamg_update_split write it so).
 * Columns hold the unnormalised vectors vt_j.
 *   nsamg_split_basis: column j of the FP64 block d_V (ldv) -> column j of d_Vs (lds), j < ncols.
 *   nsamg_gram_split:  out[0..i] = vt_j . vt_i, out[i+1..2i+1] = vt_j . w for j = 0..i (raw
 *                      products; a solve scales them by 1 / beta_j), double-FP32 per block and
 *                      FP64 across blocks, deterministic; a block whose w lies outside the
 *                      [2^-50, 2^60] window is computed in FP64 from the stored pairs.
 *   nsamg_update_split: column i+1 = w / beta_i - sum_{j<=i} c_j vt_j with c_j (device, i+1
 *                      doubles) the coefficients of the stored vectors (h_j / beta_j in a solve),
 *                      stored as a pair; *d_sumsq (device) = its squared norm; d_vin (device, n
 *                      doubles, may be NULL) receives its FP64 value.
 * d_Vs and d_w must be 16-byte aligned, lds even and lds >= n rounded up to even (INVALID_ARG
 * otherwise); 0 <= i <
 * NSAMG_MAX_RESTART and the update writes column i+1, so the block needs i+2 columns. Scratch and
 * serialisation as nsamg_gram / nsamg_update (the same two families). Asynchronous on `stream`. */
int nsamg_split_basis(int64_t n, int ncols, const double* d_V, int64_t ldv, void* d_Vs, int64_t lds, void* stream);
int nsamg_gram_split(int64_t n, int i, const void* d_Vs, int64_t lds, const double* d_w, double* d_out, void* stream);
int nsamg_update_split(int64_t n, int i, void* d_Vs, int64_t lds, const double* d_w, double beta_i, const double* d_c,
                       double* d_vin, double* d_sumsq, void* stream);

/* Allocation-free variant of nsamg_gram (the paper has no counterpart; this is a service
 * to callers). Same arguments, same results: out[0..i] = [V_i, vt]^T vt, out[i+1..2i+1] =
 * [V_i, vt]^T w. It is meant for callers that must not allocate device memory: an application
 * whose own allocator has already reserved the device memory it is allowed to use, or a
 * latency-critical loop that cannot risk entering the CUDA allocator (which may synchronise the
 * device or fail under memory pressure). Its scratch is a fixed array inside the library image
 * (about 520 KB, room for 512 blocks x 2 x 65 doubles plus a counter) that every device loading
 * the library keeps until the process exits; no cudaMalloc, cudaFree or other allocating routine
 * is called. Limit: i <= 63 (columns 0..63); larger i is rejected with NSAMG_ERR_INVALID_ARG.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) and
 * should come before any stream capture. All calls share the one array and each call clears its
 * counter first: calls that overlap on the GPU (different streams, or threads without ordering)
 * race and give wrong results, so serialise them. */
int nsamg_gram_noalloc(int64_t n, int i, const double* d_V, int64_t ldv, const double* d_w, double* d_out,
                       void* stream);

/* ||S_k||_2 for the k x k strictly lower matrix L_k (device, row-major, leading dimension ld >= k;
 * only the entries below the diagonal are read): S_k = (I + L_k^T)^-1 L_k^T, the matrix of Paige,
 * Rozloznik and Strakos that Sec. 3 uses to detect the loss of linear independence of the Krylov
 * basis (||S_k||_2 = 1 exactly when the columns of V_k are dependent). The solve computes it on the
 * last cycle's L (nsamg_stats.sk_norm); this entry runs the same kernel on caller data.
 * Method: S_k by back substitution, then power iteration on S_k^T S_k until the Rayleigh quotient
 * changes by at most 1e-15 relative (300 iterations at most); deterministic. Writes one double to
 * d_out on `stream` (asynchronous). 1 <= k <= NSAMG_MAX_RESTART, else INVALID_ARG. */
int nsamg_sknorm(const double* d_L, int ld, int k, double* d_out, void* stream);

/* Measurement probe (the paper has no counterpart): launches `blocks` x 256 threads, each
 * running 8 independent FMA chains for `iters` rounds in FP64 (fp64 = 1) or FP32 (fp64 = 0), and
 * stores one value per thread into d_sink (device, blocks x 256 elements of that type). Time the
 * launch with events on `stream`; *fma_per_launch (host, may be NULL) receives the FMA count.
 * Used to measure the FP64 and FP32 FMA rates that bound the FP64 and double-FP32 kernels. */
int nsamg_fma_probe(int fp64, int64_t iters, int blocks, void* d_sink, void* stream, double* fma_per_launch);

/* Test of the bounded grid barrier that the grid-wide fused tail (fuse_tail = 2) places between
 * its passes (the paper has none: each of its V-cycle passes is a kernel launch). One cooperative
 * launch of one 256-thread block per SM runs `rounds` barriers, each expecting the grid's blocks
 * plus `missing` arrivals; with missing > 0 no barrier can complete, and every block gives up
 * after `spin_limit` polls of about 0.1 us. On return (synchronous) *passed = barriers completed,
 * summed over blocks (rounds x SMs when missing = 0), *status = 0, or NSAMG_ERR_TIMEOUT if a
 * wait gave up. INVALID_ARG for rounds < 1, missing < 0, spin_limit < 1 or null pointers. */
int nsamg_grid_barrier_test(int rounds, int missing, unsigned spin_limit, int* passed, int* status);

/* ---- batched solves of many independent systems ----------------------------------------
 * nsamg_batch_setup: `count` host hierarchies with the same number of levels (and either all or
 * none with a coarse dense inverse) are concatenated block-diagonally: system s owns rows
 * [off_s, off_s + n_s) of every concatenated vector (nsamg_batch_offsets returns the count+1
 * offsets). Every V-cycle kernel then covers all systems in one launch; GMRES runs in lock step
 * with a separate state per system (its own beta, L, Hessenberg/Givens and stopping), each
 * system stopping on its own test. The returned handle works with nsamg_apply_vcycle and
 * nsamg_batch_solve (not nsamg_solve). Errors as nsamg_setup_hierarchy; INVALID_ARG if the
 * depths differ or the total row count exceeds INT32_MAX.
 * nsamg_batch_solve: d_b, d_x are the concatenated device vectors (x0 in, x out); `stats` (may
 * be NULL) receives `count` entries. Returns OK if every system converged, NOT_CONVERGED if some
 * did not, or the first error. Blocks until done. */
int nsamg_batch_setup(const nsamg_hierarchy_desc* hs, int count, const nsamg_params* p, void* cuda_stream,
                      nsamg_handle** out);
int nsamg_batch_solve(nsamg_handle* h, const double* d_b, double* d_x, double rtol, int maxit, nsamg_stats* stats);
int nsamg_batch_count(nsamg_handle* h);
int nsamg_batch_offsets(nsamg_handle* h, int64_t* out);

/* ---- request server (continuous batching of solves on resident hierarchies) -------------
 * nsamg_server_create: a server for the current device with a device-memory budget (bytes) for
 * solver contexts and at most `max_slots` solves in flight. A worker thread admits queued
 * requests in arrival order as soon as a slot is free and a context for the request's
 * hierarchy fits the budget (idle contexts are reused, least recently used idle contexts of
 * other hierarchies are evicted); solves of different slots run concurrently on their own
 * streams, each as one CUDA graph. Hierarchies stay owned by the caller and must outlive the
 * server's use of them; they must be set up with use_graph = 1.
 * nsamg_server_submit: queue a solve of A x = b (device arrays, valid until the request
 * completes); returns a ticket. `ready_stream` (a cudaStream_t, NULL = legacy default stream) is
 * the stream on which b and x0 were produced: the solve starts after the work queued there so far. nsamg_server_poll: NSAMG_PENDING while queued or running, else
 * the final status (the ticket is then released); `times` (may be NULL) gets submit, start and
 * completion times in seconds on the server's clock. nsamg_server_wait blocks until done.
 * nsamg_server_cancel removes a request that has not started. A request whose context can never
 * fit the budget completes with NSAMG_ERR_ADMISSION. nsamg_server_info: bytes in use, contexts,
 * running, queued. nsamg_server_destroy drops queued requests, waits for running ones and frees
 * every context. */
typedef struct nsamg_server nsamg_server;
int nsamg_server_create(size_t hbm_budget_bytes, int max_slots, nsamg_server** out);
int nsamg_server_submit(nsamg_server* s, nsamg_handle* h, const double* d_b, double* d_x, double rtol, int maxit,
                        void* ready_stream, uint64_t* ticket);
int nsamg_server_poll(nsamg_server* s, uint64_t ticket, nsamg_stats* st, double* times);
int nsamg_server_wait(nsamg_server* s, uint64_t ticket, nsamg_stats* st, double* times);
int nsamg_server_cancel(nsamg_server* s, uint64_t ticket);
int nsamg_server_info(nsamg_server* s, int64_t* out4);
void nsamg_server_destroy(nsamg_server* s);

/* ILU(0) factors of A computed on the current device by fixed-point sweeps (the iteration the
 * paper's conclusions propose for a cheaper setup): with the products l_ik u_kj (k < min(i, j))
 * of every entry of pattern(A),
 *   i > j: l_ij = (a_ij - sum_k l_ik u_kj) / u_jj,   i <= j: u_ij = a_ij - sum_k l_ik u_kj,
 * applied `sweeps` times in Jacobi fashion from l = a_ij / a_jj, u = a_ij. The exact ILU(0) is
 * the fixed point. A: host CSR (validated); lu_out: host array of nnz(A) values on A's pattern
 * (strictly lower entries = L_s, the rest = U with its diagonal). Blocks on `stream`. */
int nsamg_ilu0_fixed_point(const nsamg_csr* A, int sweeps, double* lu_out, void* stream);

/* ---- Ruge-Stuben setup on the GPU (Sec. 5.1) ------------------------------------------------
 * The paper's conclusions name a GPU setup as the next step; these calls build the hierarchy the
 * solve phase consumes with every step on the current device:
 *   strength  S_i = { j != i : m(a_ij) >= theta max_{k != i} m(a_ik) }, m = |.| (strength_mode 0,
 *             as printed in Sec. 5.1) or -(.) (strength_mode 1, the classical sign-aware form);
 *   PMIS      (Sec. 5.1) weights lambda_i = |S^T_i| + u_i, u_i the top 53 bits of one SplitMix64
 *             step from the state seed_l ^ (0xA24BAED4963EE407 (i + 1)), seed_l = seed + 7919 (l + 1)
 *             for level l; rounds select the undecided points that no undecided point of
 *             S_i u S^T_i outranks in (lambda, index); undecided points that strongly depend on a
 *             new C-point become F; points that influence no one start as F; F-points left without
 *             a strong C-neighbour are then promoted to C (they influence no point, so the
 *             order of promotion does not matter);
 *   BAMG-direct interpolation, closed form of eq. (bamgdir) with f = 1:
 *             w_ij = -(a_ij + beta_i / n_{C_i^s}) / (a_ii + sum_{k weak} a_ik), beta_i the sum of
 *             the strong F-couplings; C rows are unit rows;
 *   MM-ext    (interp = 1, Sec. 5.1) W = -[(D_FF + D_gamma)^-1 (A^s_FF + D_beta)] [D_beta^-1 A^s_FC],
 *             D_beta = diag(A^s_FC 1), D_gamma = diag(A^w_FF 1 + A^w_FC 1) (weak couplings), P = [W; I]
 *             in the original ordering; an F-point with beta = 0 adds no distance-two path;
 *   Galerkin  R = P^T, A_c = R (A P) (Sec. 5, eq. A_k); each entry of a product is summed in the
 *             order of the left operand's row, with products and sums rounded separately;
 *   ILU(0)    `ilu_sweeps` fixed-point sweeps (as nsamg_ilu0_fixed_point) on every level l < L-1
 *             whose bit is set in `ilu_levels`, stored in the row-scaled LDU form of
 *             nsamg_level_desc (ilu_form 0, U_s = diag(U)^-1 strict_upper(U), dinv = 1/u_ii);
 *   coarse    dense inverse of the coarsest operator by Gauss-Jordan with partial pivoting when it
 *             has at most `direct_max` rows.
 * Coarsening stops when a level has at most `coarse_max` rows, at `max_levels` levels, or when a
 * step keeps no point or at least 90% of them. */
typedef struct {
  double theta;          /* strength threshold, 0 <= theta <= 1 (default 0.25)                 */
  int32_t strength_mode; /* 0: |a_ij|, 1: -a_ij                                                */
  int32_t max_levels;    /* >= 1 (default 25)                                                   */
  int32_t coarse_max;    /* >= 1 (default 512)                                                  */
  int32_t direct_max;    /* 0..8192 (default 512)                                               */
  uint64_t seed;         /* PMIS seed (default 0)                                               */
  uint64_t ilu_levels;   /* bit l: ILU(0) factors on level l (default 1: the finest level)      */
  int32_t ilu_sweeps;    /* fixed-point sweeps, >= 0 (default 3)                                */
  int32_t interp;        /* 0: BAMG-direct (default), 1: MM-ext                                 */
} nsamg_amg_options;

typedef struct nsamg_amg nsamg_amg;

void nsamg_amg_default_options(nsamg_amg_options* o);

/* Build the hierarchy of A (host CSR, validated like nsamg_setup_hierarchy's input: square,
 * sorted columns, nonzero diagonal, finite values) on the current device, on `cuda_stream`.
 * Blocks until done. The hierarchy lives in device memory owned by *out.
 * Errors: INVALID_ARG (null pointer, option out of range), BAD_MATRIX (validation; a row whose
 * interpolation is undefined; a singular coarsest operator; a matrix beyond 2^31 - 1 entries),
 * OOM, CUDA. On error *out is NULL. */
int nsamg_amg_build(const nsamg_csr* A, const nsamg_amg_options* opt, void* cuda_stream, nsamg_amg** out);
int nsamg_amg_num_levels(const nsamg_amg* g);
/* Level l: rows, nonzeros of A_l, coarse points chosen on it (0 on a level that was not
 * coarsened) and PMIS rounds taken. Any output pointer may be NULL. */
int nsamg_amg_level_info(const nsamg_amg* g, int l, int32_t* n, int64_t* nnz, int32_t* nc, int32_t* pmis_rounds);
/* Host copies of level l's splitting: cf (n_l entries: coarse index, or -1 for F) and the strength
 * flags (nnz(A_l) bytes, 1 = strong, in CSR order). Either pointer may be NULL. INVALID_ARG on a
 * level that was not coarsened. */
int nsamg_amg_level_splitting(const nsamg_amg* g, int l, int32_t* cf, uint8_t* strong);
/* Host copy of the whole hierarchy as a nsamg_hierarchy_desc; the arrays are owned by g and stay
 * valid until the next export or nsamg_amg_destroy. */
int nsamg_amg_export(nsamg_amg* g, nsamg_hierarchy_desc* out);
/* A solver handle for the GPU-built hierarchy, formed on the device without a host round trip:
 * the solve-phase arrays (D^-1, l1 diagonal, scaled triangles, plain SELL copies of near-uniform
 * matrices, transfers, ILU(0) factors of the levels the smoother uses, coarse inverse) are derived
 * from g's device operators by kernels, with the same arithmetic as nsamg_setup_hierarchy on the
 * exported hierarchy (with fixed threads per row the two handles give bitwise equal solves;
 * matrices that are not near-uniform get no sorted SELL copy here). The handle owns its own
 * copies; g may be destroyed afterwards. Blocks until done.
 * Errors: INVALID_ARG (null pointer, parameter out of range), BAD_MATRIX (a level operator with a
 * missing or zero diagonal or a non-finite entry), OOM, CUDA. On error *out is NULL. */
int nsamg_amg_setup_solver(nsamg_amg* g, const nsamg_params* p, void* cuda_stream, nsamg_handle** out);
void nsamg_amg_destroy(nsamg_amg* g);

/* Matrix layout chosen for a level's operator (diagnostic): 0 = the SELL-32 copy (chunks of 32
 * rows stored column-major, one thread per row; natural row order when that pads by <= 3%, else
 * rows sorted by length inside windows of 4096 rows), else the number of threads per row of the
 * CSR kernel. For an FP32 V-cycle handle, the FP32 copy of the level's operator. */
int nsamg_level_group(nsamg_handle* h, int level);

/* Kernel launches in one Arnoldi step (V-cycle, SpMV, Gram, update). A solve launches
 * 1 + iters * launches_per_step + 2 * (restarts + 1) kernels. */
int nsamg_launches_per_step(nsamg_handle* h);

void nsamg_destroy(nsamg_handle* h);
const char* nsamg_status_str(int status);
const char* nsamg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NSAMG_H */
