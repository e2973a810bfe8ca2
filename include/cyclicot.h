/*
 * cyclicot.h -- C ABI of the GB300 (sm_103a) library for optimal transport
 * with cyclic symmetry (Takeda, Akagi, Marumo, Niwa, AAAI-24, arXiv 2311.13147).
 *
 * Problem (Sec. 3.2, Eq. problem_ROT):  min_T <C,T> + sum_ij phi(T_ij)
 * subject to T 1 = a, T^T 1 = b, with phi = 0 on x >= 0 (LOT, Eq.
 * reg_for_original_OT) or phi(x) = eps * x (log x - 1) (EROT, Eq.
 * reg_for_entropy_ROT; the paper calls eps "lambda").
 *
 * Cyclic symmetry (Assumption 1, Sec. 4): the full size is n = N * m, the
 * marginals are N copies of base blocks, a = (alpha; ...; alpha), and the cost
 * is block-circulant, block (r, c) = C_{(c - r) mod N}
 * (Eq. blkstr_cost).  This library takes the first block row
 * C_base[k] = C[0:m, k*m:(k+1)*m] as a dense float array [N][m][m] (row-major,
 * k slowest), or the base point coordinates when C_k[i][j] = |x_i - R^k y_j|^2
 * with R the rotation by 2*pi/N.
 *
 * Letters: the paper's d (full size) is n here, its n (cyclic order) is N.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All array arguments are DEVICE pointers owned by the caller (for example
 *   from PyTorch tensors).  float arrays must be 16-byte aligned.  The library
 *   never allocates memory: scratch space comes from the caller's workspace
 *   (size from ot_workspace_bytes), and nothing is kept between calls.
 * - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *   stream.  Every call is asynchronous with respect to the host: results,
 *   including the ot_result record, are valid after the stream is
 *   synchronised.
 * - Marginal inputs a_base, b_base (and a, b for full problems) may have any
 *   positive mass; they are normalised internally (sums in FP64).  Every entry
 *   must be > 0 (log-domain iterations); a zero or non-finite entry makes the
 *   solver report OT_ERR_ARG in ot_result.status.
 * - Return value: OT_OK when the work was enqueued; otherwise an error code
 *   for problems detectable on the host (null pointer, bad size, too small a
 *   workspace, CUDA launch failure).  Errors found on the device (divergence,
 *   non-finite values, an expired wait) are written to ot_result.status.
 * - No entry point aborts, traps or exits the process.
 */
#ifndef CYCLICOT_H
#define CYCLICOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define OT_OK                 0
#define OT_ERR_ARG            1   /* null pointer, m <= 0, N <= 0, eps <= 0, bad mode       */
#define OT_ERR_NOT_DIVISIBLE  2   /* full size n is not a multiple of the cyclic order N    */
#define OT_ERR_NOT_CONVERGED  3   /* max_iter reached; outputs hold the last iterate         */
#define OT_ERR_TIMEOUT        4   /* a bounded device-side wait expired (grid barrier)       */
#define OT_ERR_NONFINITE      5   /* NaN / Inf met in the iteration                          */
#define OT_ERR_CUDA           6   /* a CUDA runtime call failed                              */
#define OT_ERR_WORKSPACE      7   /* workspace pointer NULL or smaller than required         */
#define OT_ERR_UNSUPPORTED    8   /* size or mode outside what this build supports           */

/* ---- modes ----------------------------------------------------------- */
#define OT_MIN                0   /* LOT fold, Theorem 1                                     */
#define OT_SOFTMIN            1   /* EROT fold, Eq. def_Kij in log form                      */

#define OT_PLAN_LOT           0   /* unfold Theorem 1's S* by the smallest argmin            */
#define OT_PLAN_EROT          1   /* unfold Theorem 2's potentials                           */

#define OT_ADJ_ENVELOPE       0   /* gradient from the converged potentials                 */
#define OT_ADJ_UNROLLED       1   /* reverse pass through a fixed number of iterations        */

/* stopping norms (ot_options.stop_norm) of ot_sinkhorn_reduced / _full:
 * L1_FULL: sum over the n full rows of |T 1 - a| (the reduced solver's
 *          N sum_i |S 1 - alpha|_i), compared with tol_l1;
 * L2_ROW:  ||S 1 - alpha||_2 of the problem as solved (mass 1/N marginals for
 *          the reduced problem, unit mass for the full one): the Stage-1 rule
 *          of Algorithm 3 (App. F); ot_result.marg_l1 then holds this norm.
 * The batch and kernel-domain solvers use L1_FULL only. */
#define OT_STOP_L1_FULL       0
#define OT_STOP_L2_ROW        1

#define OT_FP32_LOG           0   /* FP32 log-domain iterations (default)                    */
#define OT_BF16_KERNEL_POLISH 1   /* BF16 kernel-domain GEMM iterations, then FP32 polish    */

/* ops for ot_workspace_bytes */
#define OT_OP_SINKHORN_REDUCED 0
#define OT_OP_SINKHORN_FULL    1
#define OT_OP_VALUE_AND_GRAD   2
#define OT_OP_UNROLLED         3

typedef struct {
    float eps;                      /* regulariser (> 0)                                   */
    double tol_l1;                  /* stop when the full-scale row L1 error <= tol_l1     */
    int max_iter;                   /* iteration cap (>= 1)                                */
    int check_every;                /* test the stopping rule every k iterations (>= 1)    */
    int precision;                  /* OT_FP32_LOG (the only value ot_sinkhorn_* take)     */
    int warm_start;                 /* 1: start from the g passed in (f is recomputed)     */
    unsigned long long timeout_ns;  /* limit of each device-side wait; 0 = 10 s            */
    int tile_override;              /* 0; batch solver: a configuration code (autotune)    */
    int debug_flags;                /* 0 in normal use.
                                       bit 0 (OT_DEBUG_WITHHOLD_ARRIVAL), fault injection:
                                       block 0 never arrives at the first grid barrier,
                                       so the other blocks' bounded waits expire and the
                                       solve reports OT_ERR_TIMEOUT.
                                       bit 1 (OT_DEBUG_TRACE), tracing: block 0 records
                                       %globaltimer stamps (ns) per sweep t < 256 in the
                                       last 16 KB of the workspace, 8 uint64 per sweep:
                                       [0] sweep start, [1] row phase done, [2] after the
                                       first grid barrier, [3] column phase done.
                                       bit 2 (OT_DEBUG_NO_CLUSTER): do not use the
                                       ring or bulk-reduce solvers; use the two-barrier
                                       FP64-partial one (comparison runs).
                                       bit 3 (OT_DEBUG_NO_RING): do not use the ring
                                       solvers (per-thread copy ring, FP32 sweep); use
                                       the FP64 bulk-reduce one (comparison runs).      */
    int stop_norm;                  /* OT_STOP_L1_FULL (default) or OT_STOP_L2_ROW          */
} ot_options;

#define OT_DEBUG_WITHHOLD_ARRIVAL 1
#define OT_DEBUG_TRACE            2
#define OT_DEBUG_NO_CLUSTER       4
#define OT_DEBUG_NO_RING          8

/* Device-written outcome of one solve.  64 bytes, naturally aligned. */
typedef struct {
    int iters;              /* completed iterations of the returned state               */
    int status;             /* OT_OK / OT_ERR_*                                          */
    double marg_l1;         /* full-scale row L1 error sum_i |(T 1)_i - a_i| of the state  */
    double marg_l2_col;     /* ||T^T 1 - b||_2 (filled by ot_value_and_grad)             */
    double value;           /* regularised objective of the full problem (value_and_grad)  */
    double transport_cost;  /* <C, T> of the full problem (value_and_grad)              */
    double marg_l1_col;     /* full-scale column L1 error (value_and_grad)               */
    double reserved[2];
} ot_result;

/* ---- entry points ------------------------------------------------------ */

/* Library version string, e.g. "cyclicot 0.1 sm_103a". */
const char* ot_version(void);

/* Human-readable name of a status code (static storage). */
const char* ot_status_string(int status);

/* Bytes of workspace that `op` needs for a problem of block size m (reduced
 * ops) or full size n (full ops), cyclic order N.  Returns 0 for a bad op. */
size_t ot_workspace_bytes(int op, int m_or_n, int N, const ot_options* opt);

/*
 * ot_fold_cost -- fold the N cost blocks into the m x m reduced cost.
 *
 *  mode = OT_MIN (Theorem 1, Eq. definition_G):
 *      G[i][j] = min_k C_k[i][j],  kstar[i][j] = smallest k attaining it
 *      (Eq. optimal_solution_problem_CLOT takes the smallest argmin).  The
 *      comparison is exact: results are bit-identical to any exact min.
 *  mode = OT_SOFTMIN (Sec. 5.4, Eq. def_Kij):
 *      G[i][j] = -eps * log K_ij,  K_ij = sum_k exp(-C_k[i][j] / eps),
 *      computed as cmin - eps * log sum_k exp(-(C_k[i][j] - cmin)/eps).
 *      The reduced EROT problem is then a plain m x m EROT on G with
 *      marginals of mass 1/N; no log N term enters the fold.  kstar unused.
 *
 *  Cost source: C_base [N][m][m] if non-NULL; else points x [m][2] (sources)
 *  and y [m][2] (targets), C_k[i][j] = |x_i - R^k y_j|^2, R = rotation by
 *  2*pi/N (computed in FP32).
 *  Outputs: G [m][m] float; kstar [m][m] uint8 (OT_MIN only, N <= 255).
 *  Returns OT_ERR_ARG (m or N <= 0, G NULL, an unknown mode, eps <= 0 with
 *  OT_SOFTMIN, no cost source) or OT_ERR_UNSUPPORTED (OT_MIN with N > 255: k*
 *  is one byte) before anything is enqueued, OT_ERR_CUDA on a failed launch.
 */
int ot_fold_cost(int mode, int m, int N, const float* C_base, const float* x,
                 const float* y, float eps, float* G, uint8_t* kstar, void* stream);

/*
 * ot_sinkhorn_reduced -- cyclic Sinkhorn (Algorithm 2) on the folded cost.
 *
 * Runs the alternating closed-form dual updates of Eq.
 * optimal_f_sinkhorn_logdomain in the log domain on the m x m cost G from
 * ot_fold_cost(OT_SOFTMIN):
 *     w_i = eps log alpha_i - eps LSE_j((z_j - G_ij)/eps)   (row update)
 *     z_j = eps log beta_j  - eps LSE_i((w_i - G_ij)/eps)   (column update)
 * from z = 0 (q = 1), until the full-scale row L1 error
 * N * sum_i |(S 1)_i - alpha_i| <= opt->tol_l1, where S = sum_k T_k.
 *
 *  a_base, b_base [m]: base marginal blocks (any positive mass; alpha =
 *      a_base / (N * sum a_base)).
 *  w, z [m] double, out: potentials of the returned state for marginals of
 *      mass 1/N (the paper's w, z; T_ijk = exp((w_i + z_j - C_ijk)/eps)).
 *      With opt->warm_start = 1, z is read as the starting point.
 *  out: device ot_result (iters, status, marg_l1).
 *  workspace: >= ot_workspace_bytes(OT_OP_SINKHORN_REDUCED, m, N, opt).
 */
int ot_sinkhorn_reduced(int m, int N, const float* a_base, const float* b_base, const float* G,
                        const ot_options* opt, double* w, double* z, ot_result* out,
                        void* workspace, size_t ws_bytes, void* stream);

/*
 * ot_sinkhorn_reduced_static -- ot_sinkhorn_reduced without a caller workspace.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory where they call the solver (a plugin inside a
 * framework that owns the device allocator, a loop that must not allocate
 * after start-up).  Arguments and results are those of ot_sinkhorn_reduced;
 * the scratch space comes from a 4 MiB array compiled into the library (one
 * per device, held until the process exits).  Each call checks
 * ot_workspace_bytes(OT_OP_SINKHORN_REDUCED, m, N, opt) against the array
 * (the need grows with m and the device's SM count; every m <= 4096 fits on a
 * 152-SM GB300) and returns OT_ERR_UNSUPPORTED, launching nothing, when it
 * does not fit.  All calls on a device share the array (each call clears what
 * must start at zero), so calls that overlap on the GPU race.  The first call
 * on a device looks up the array's address with cudaGetSymbolAddress on the
 * current device: make it before any stream capture, and do not reset the
 * device afterwards (the stored address would be stale).  Nothing here
 * allocates memory.
 */
int ot_sinkhorn_reduced_static(int m, int N, const float* a_base, const float* b_base, const float* G,
                               const ot_options* opt, double* w, double* z, ot_result* out, void* stream);

/*
 * ot_sinkhorn_full -- plain Sinkhorn on the full n x n problem (the
 * comparison; Algorithm 3 Stage 2), same iteration and stopping rule.
 *
 *  a, b [n]: marginals (normalised internally).
 *  C [n][n] float if non-NULL; else X [n][2], Y [n][2] and the cost
 *      C_ij = |X_i - Y_j|^2 is computed on the fly (never stored).
 *  f, g [n] double, out (g read first when opt->warm_start = 1, e.g. the
 *      N-fold concatenated Stage-1 potentials of Algorithm 3).
 */
int ot_sinkhorn_full(int n, const float* a, const float* b, const float* C,
                     const float* X, const float* Y, const ot_options* opt,
                     double* f, double* g, ot_result* out,
                     void* workspace, size_t ws_bytes, void* stream);

/*
 * ot_unfold_plan -- reconstruct the block-circulant plan.
 *
 *  mode = OT_PLAN_LOT (Theorem 1): T_k[i][j] = S[i][j] if k == kstar[i][j]
 *      else 0.  S_or_w = S [m][m] float (an optimal reduced plan), kstar from
 *      ot_fold_cost(OT_MIN); z, C_base, x, y unused.
 *  mode = OT_PLAN_EROT (Algorithm 2's reconstruction, Theorem 2):
 *      T_k[i][j] = exp((w_i + z_j - C_k[i][j]) / eps); S_or_w = w (double
 *      [m], cast), z [m] double; cost from C_base or from x, y as in
 *      ot_fold_cost.
 *  dense = 0: T is the first block row [N][m][m] (T_0..T_{N-1});
 *  dense = 1: T is the n x n matrix, T[r*m+i][c*m+j] = T_{(c-r) mod N}[i][j]
 *      (Lemma 1, Eq. blkstr_optimal_solution).  Index map is exact.
 *  Returns OT_ERR_ARG (m or N <= 0, S_or_w or T NULL, an unknown mode;
 *  OT_PLAN_LOT without kstar or with N > 255; OT_PLAN_EROT without z, with
 *  eps <= 0 or without a cost source) or OT_ERR_CUDA.
 */
int ot_unfold_plan(int mode, int m, int N, const void* S_or_w, const double* z,
                   const float* C_base, const float* x, const float* y,
                   const uint8_t* kstar, float eps, int dense, float* T, void* stream);

/*
 * ot_value_and_grad -- objective, marginal norms and gradients of the EROT
 * value through the reduced problem.
 *
 *  value (out->value): N * [ sum_ijk C_ijk T_ijk + eps T_ijk (log T_ijk - 1) ]
 *      (Eq. problem_CROT times N, Sec. 5.1), out->transport_cost
 *      N * sum_ijk C_ijk T_ijk, full-scale row / column L1 and column L2
 *      marginal errors; all reductions in FP64.
 *  adjoint = OT_ADJ_ENVELOPE: gradients from Theorem 2's dual at (w, z):
 *      d_a[m] = dV/da_base = (w - <w,a_base>/s)/s, s = sum a_base (likewise
 *      d_b with z); d_C [N][m][m] = N * T_k (if C_base given), or
 *      d_x, d_y [m][2] = 2N sum T_ijk (x_i - R^k y_j), 2N sum T_ijk
 *      (y_j - R^-k x_i) (if points given).  Any gradient pointer may be NULL.
 *  adjoint = OT_ADJ_UNROLLED: gradients of V_T = N(<w_T,alpha> + <z_T,beta>)
 *      - eps after `unroll_iters` iterations from z = 0, by a reverse pass
 *      that re-reads the folded cost G (which must be passed) and the
 *      checkpointed potentials; w, z are ignored (the forward pass is rerun).
 */
int ot_value_and_grad(int m, int N, const float* a_base, const float* b_base,
                      const float* C_base, const float* x, const float* y,
                      const float* G, const double* w, const double* z, float eps,
                      int adjoint, int unroll_iters, ot_result* out,
                      float* d_a, float* d_b, float* d_C, float* d_x, float* d_y,
                      void* workspace, size_t ws_bytes, void* stream);

/* ---- batches of independent cyclic problems (uneven m and N) ------------ */

/* One problem of a batch.  48 bytes. */
typedef struct {
    int m;              /* block size                                                      */
    int N;              /* cyclic order                                                    */
    float eps;          /* regulariser                                                     */
    int ld;             /* row stride of its folded cost: multiple of 4, m <= ld <= 8192;
                           the pad entries [m, ld) of each row must be finite (the fold
                           writes 0)                                                       */
    long long g_off;    /* offset (floats, multiple of 4) of its cost G [m][ld] in G_all    */
    long long v_off;    /* offset (elements) of its vectors in a_all, b_all, w_all, z_all   */
    long long x_off;    /* offset (points) of its base source points in the point buffer   */
    long long y_off;    /* offset (points) of its base target points in the point buffer   */
} ot_problem_desc;

/* Workspace bytes of a batch of `count` problems with sum of m equal to total_m. */
size_t ot_batch_workspace_bytes(int count, long long total_m);

/*
 * ot_batch_prepare -- copy the problem table into the workspace (outside any
 * stream capture).  descs is HOST memory (count entries); it is not read
 * after the call returns.  The header the solver reads (sizes, and the number
 * of problems of each rows-per-chunk class) is written here.
 */
int ot_batch_prepare(const ot_problem_desc* descs, int count, void* workspace, size_t ws_bytes, void* stream);

/*
 * ot_batch_fold -- Eq. def_Kij soft-min fold for every problem of a prepared
 * batch, cost from points: C_k[i][j] = |x_i - R^k y_j|^2, R the rotation by
 * 2*pi/N (points: float2 array, offsets from the descriptors).  Writes each
 * problem's G into G_all at g_off with row stride ld.
 */
int ot_batch_fold(int count, const float* points, float* G_all, void* workspace, size_t ws_bytes, void* stream);

/*
 * ot_batch_solve -- cyclic Sinkhorn (Algorithm 2) on every problem of a
 * prepared batch in two persistent cooperative launches (capturable in a CUDA
 * graph: it only enqueues kernels and memsets): one for the problems whose
 * rows fill three float4 slots per thread of their group (processed three
 * rows per group at a time), one for the others (two rows at a time); a
 * launch without problems of its kind returns at once.  Each sweep re-balances the
 * rows of the still-active problems over the blocks; a problem leaves the
 * batch when its full-scale row L1 error <= opt->tol_l1 (its state is then
 * frozen) or after opt->max_iter iterations.  opt->eps is ignored (per
 * problem eps in the descriptors).  Outputs per problem: w, z (mass-1/N
 * convention, as ot_sinkhorn_reduced) at v_off, and results[p] (device array
 * of `count` ot_result: iters, status, marg_l1).  total_m = max over problems
 * of v_off + m (the length of the vector buffers), as given to prepare.
 * opt->tile_override selects a launch configuration: 0 = default (tight
 * thread groups, convergence tested every opt->check_every iterations), or a
 * code returned by ot_batch_autotune (1..6).  With a
 * cadence k > 1 a problem stops at the first multiple of k whose state meets
 * the tolerance.
 * G_all must be 16-byte aligned (cost rows are streamed with bulk copies);
 * otherwise OT_ERR_ARG.  A copy or grid barrier that does not complete within
 * opt->timeout_ns (0: 10 s) ends that launch with OT_ERR_TIMEOUT in the
 * results of its problems (iters = -1).  The problems of one prepared workspace must not be
 * solved on two streams at once.
 */
int ot_batch_solve(int count, long long total_m, const float* G_all, const float* a_all, const float* b_all,
                   const ot_options* opt, double* w_all, double* z_all, ot_result* results, void* workspace,
                   size_t ws_bytes, void* stream);

/*
 * ot_batch_autotune -- choose the batch solver's launch configuration for a
 * prepared batch on the current device (no counterpart in the paper: an
 * implementation choice).  Times, on `stream`, the two group-size policies
 * (the smallest thread group covering a row, or one size larger) over 4 full
 * sweeps, then the convergence-check cadences 1, 2, 4 with complete solves
 * under opt's tolerance; returns the fastest code in *config_out (pass it as
 * ot_options.tile_override to ot_batch_solve).  ms_out (host, 5 floats, may
 * be NULL) receives the measured times.  The
 * result is cached per (device, problem table, tol, max_iter): a repeated call
 * returns the cached code without launching anything.  Otherwise the outputs
 * (w, z, results) are those of a complete solve with the chosen code.  Blocks
 * the calling thread; must not be called while `stream` is being captured
 * (OT_ERR_ARG).
 */
int ot_batch_autotune(int count, long long total_m, const float* G_all, const float* a_all, const float* b_all,
                      const ot_options* opt, double* w_all, double* z_all, ot_result* results, void* workspace,
                      size_t ws_bytes, void* stream, int* config_out, float* ms_out);

/* ---- Algorithm 3 (two-stage, approximate cyclic symmetry) ------------------ */

/*
 * ot_first_block_row -- C_base[k][i][j] = C[i][k m + j] for the full cost C
 * [n][n] (n = N m, FP32 row-major): the blocks that define K in Algorithm 3's
 * Stage 1 (Eq. def_Kij).  C_base: [N][m][m] FP32.  Device pointers, async.
 */
int ot_first_block_row(int m, int N, const float* C, float* C_base, void* stream);

/*
 * ot_block_average -- out_i = (1/N) sum_k v[k m + i] (Algorithm 3, Stage 1:
 * the reduced marginals of an approximately symmetric input; FP64 sum).
 * v: [N m] FP32, out: [m] FP32.  Device pointers, async.
 */
int ot_block_average(int m, int N, const float* v, float* out, void* stream);

/*
 * ot_tile_potentials -- g[k m + j] = z[j] for k < N (Algorithm 3, Stage 2
 * initialisation: the N-fold concatenation of the Stage-1 potential), to pass
 * as the warm start of ot_sinkhorn_full.  z: [m] FP64, g: [N m] FP64.
 */
int ot_tile_potentials(int m, int N, const double* z, double* g, void* stream);

/* ---- form 1: BF16 kernel-domain iterations on the tensor cores ----------- */

/* Workspace bytes of ot_kdomain_solve for block size m (0 if m is out of range). */
size_t ot_kdomain_workspace_bytes(int m);

/*
 * ot_kdomain_solve -- Algorithm 2 in scaling form (Eq.
 * optimal_f_sinkhorn_logdomain exponentiated: U = alpha ./ (K V),
 * V = beta ./ (K^T U), K = exp(-G / eps)) for nrhs <= 64 histogram pairs that
 * share one folded cost G.  K, K^T (tile-major) and the scalings are BF16
 * operands of tcgen05 tensor-core products with FP32 accumulation; each
 * product applies its scaling update in its own epilogue, and the scalings
 * are kept in FP32 between products.  Runs exactly `iters` iterations from V = 1 (no
 * stopping rule: BF16 bounds the reachable accuracy near 1e-3; polish the
 * result with ot_batch_solve, warm-started from z).
 *  G: [m][ld] FP32 device, ld >= m.  a_hist, b_hist: [nrhs][m] FP32 device,
 *     positive entries (each pair is normalised to unit mass).
 *  z_out: [nrhs][m] FP64 device, eps ln V (the column potential of the
 *     unit-mass reduced problem; a zero scaling maps to eps ln 1e-37).
 *  row_err: NULL or [iters][64] FP32 device: entry [t][n] is the L1 row
 *     marginal error of pair n before iteration t's row update (the state after
 *     t column updates).
 *  m <= 16384 (padded internally to a multiple of 128).  Asynchronous; a
 *  device wait that expires is reported by ot_kdomain_status.
 */
int ot_kdomain_solve(int m, const float* G, int ld, float eps, int nrhs, const float* a_hist, const float* b_hist,
                     int iters, double* z_out, float* row_err, void* workspace, size_t ws_bytes, void* stream);

/* Error flag of the last ot_kdomain_solve on `workspace` (blocks on stream). */
int ot_kdomain_status(const void* workspace, int m, int* status, void* stream);

/*
 * ot_kdomain_product -- the tensor-core product used by ot_kdomain_solve:
 * Dt[n][i] = sum_k A[i][k] X[n][k] for n < 64, i < mp; A [mp][mp] BF16,
 * X [64][mp] BF16, Dt [64][mp] FP32 (device, 16-byte aligned; mp a multiple
 * of 128, <= 16384; A row-major).  The reduction is split over the CTAs of
 * a thread-block cluster and summed in distributed shared memory, so no
 * partial product reaches global memory.  workspace: >=
 * ot_kdomain_workspace_bytes(mp) bytes, 256-byte aligned (kept for the
 * interface; the product needs none of it).  Blocks until done; returns
 * OT_ERR_TIMEOUT if a device wait expired.
 */
int ot_kdomain_product(int mp, const void* A, const void* X, float* Dt, void* workspace, size_t ws_bytes,
                       void* stream);

/* ---- C-SROT: a strongly convex regulariser other than the entropy -------- */

/* Workspace bytes of ot_srot_reduced (0 if N m > 8192 or a size is <= 0). */
size_t ot_srot_workspace_bytes(int m, int N);

/*
 * ot_srot_reduced -- Sec. 5.3 / Theorem 2 with the squared-L2 regulariser
 * phi(x) = (lambda/2) x^2 on x >= 0: alternating minimisation of the reduced
 * dual (Eq. dual_problem_cyclic_ROT), whose coordinate equations
 * sum_{k,j} (phi*)'(w_i + z_j - C_ijk) = alpha_i (Eq.
 * derivative_of_objective_function = 0, (phi*)'(y) = max(y, 0) / lambda) are
 * solved exactly (Newton on the piecewise-linear left side); the optimal plan
 * is T_ijk = max(w_i + z_j - C_ijk, 0) / lambda (Eq. optimality_condition).
 *  C_base: [N][m][m] FP32 device (the first block row).  N = 1 is the plain
 *     full problem.  N m <= 8192.
 *  a_base, b_base: [m] FP32 device, positive; normalised internally so that
 *     alpha, beta have mass 1/N.
 *  opt: eps is lambda; tol_l1 (full-scale row L1 of the returned state),
 *     max_iter, timeout_ns, warm_start (z holds the starting column potential).
 *  w, z: [m] FP64 device outputs, the dual potentials of the mass-1/N reduced
 *     problem.
 *  out: iters, status, marg_l1 (row L1), value = N sum (C T + lambda T^2 / 2),
 *     transport_cost = N sum C T (full scale); reserved[1] = 5.
 *  workspace >= ot_srot_workspace_bytes(m, N), 256-byte aligned.  Asynchronous.
 * Returns OT_ERR_ARG / OT_ERR_UNSUPPORTED / OT_ERR_WORKSPACE / OT_ERR_CUDA at
 * launch; device-side outcomes are reported in out->status.
 */
int ot_srot_reduced(int m, int N, const float* a_base, const float* b_base, const float* C_base,
                    const ot_options* opt, double* w, double* z, ot_result* out, void* workspace, size_t ws_bytes,
                    void* stream);

/* ---- C-LOT: the small linear program of Theorem 1 ----------------------- */

/* Workspace bytes of ot_lot_reduced for `count` problems of size m (0 if m > 5120 or a size is <= 0). */
size_t ot_lot_workspace_bytes(int count, int m);

/*
 * ot_lot_reduced -- exact solve of the small LOT of Theorem 1 (Eq.
 * small_problem_CLOT): min <G, S> subject to S 1 = alpha, S^T 1 = beta,
 * S >= 0, by the network simplex that Sec. 5.2 names for it (primal network
 * simplex on the complete bipartite graph; artificial-root start, block
 * pricing, the strongly-feasible-tree leaving rule).  Its value times N is the
 * value of the full C-LOT (Theorem 1 with mass 1/N blocks; the N block rows of
 * the full plan are alike); ot_unfold_plan(OT_PLAN_LOT) turns S into the
 * full plan (Eq. optimal_solution_problem_CLOT).  One thread block, or one
 * cluster of them, per problem; `count` problems of the same m in one launch.
 *  G: [count][m][m] FP32 device, finite (ot_fold_cost(OT_MIN) output).
 *  a_base, b_base: [count][m] FP32 device, >= 0 with positive sums; normalised
 *     internally so that alpha, beta have mass 1/N.
 *  opt: max_iter is the pivot cap per problem (>= 1); timeout_ns bounds each
 *     wait between the CTAs that share one problem (0 = 10 s; an expired wait
 *     ends that problem with OT_ERR_TIMEOUT); debug_flags bit 2
 *     (OT_DEBUG_NO_CLUSTER) keeps one thread block per problem, bit 0
 *     (OT_DEBUG_WITHHOLD_ARRIVAL, failure-detection tests) makes the second CTA
 *     of each cluster withhold its first candidate, so the owner's wait expires.  When the
 *     launch fits, each problem gets a thread-block cluster of 2, 4 or 8 CTAs
 *     that price separate parts of a wider block of arcs (one owns the tree);
 *     the other fields are not used.
 *  S: [count][m][m] FP32 device output, the optimal basic plan (at most 2m - 1
 *     nonzeros per problem; the flows are kept in FP64 while pivoting).
 *  u, v: [count][m] FP64 device outputs, optimal duals: u_i + v_j <= G_ij,
 *     with equality where S_ij > 0, normalised to u_0 = 0.  The pivots run on
 *     integer costs rint(G_ij 2^k), 2^k the largest power of two with
 *     max |G| 2^k < 2^30, so these hold to 2^-k (about 1e-9 max |G|) and the
 *     plan is optimal to 2^-k per unit of mass; reduced costs are exact.
 *  out: [count] device results: iters = pivots, status, value = transport_cost
 *     = N <G, S> (full scale, from the FP64 flows), reserved[0] = N (<alpha, u>
 *     + <beta, v>) (equal to value at the optimum), marg_l1 / marg_l1_col /
 *     marg_l2_col the full-scale marginal errors of the returned FP32 S,
 *     reserved[1] = 6.  status OT_ERR_ARG for a negative or
 *     non-finite entry or a zero sum (S, u, v are then NaN),
 *     OT_ERR_NOT_CONVERGED when the pivot cap was reached (S then holds the
 *     flows of the last basis on the original arcs; mass still on the
 *     artificial start arcs leaves its marginals short, see marg_l1).
 *  workspace >= ot_lot_workspace_bytes(count, m), 256-byte aligned.
 *  Asynchronous.  Returns OT_ERR_ARG / OT_ERR_UNSUPPORTED (m > 5120) /
 *  OT_ERR_WORKSPACE / OT_ERR_CUDA at launch.
 */
int ot_lot_reduced(int count, int m, int N, const float* a_base, const float* b_base, const float* G,
                   const ot_options* opt, float* S, double* u, double* v, ot_result* out, void* workspace,
                   size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CYCLICOT_H */
