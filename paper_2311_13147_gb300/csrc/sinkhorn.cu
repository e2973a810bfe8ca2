// Log-domain Sinkhorn on an M x Ncol cost: the cyclic Sinkhorn of Algorithm 2
// (on the folded m x m cost) and the plain Sinkhorn of Algorithm 3 Stage 2
// (on the full n x n cost) share this solver.
//
// Iteration (Eq. optimal_f_sinkhorn_logdomain, in log2 units phi = f/(eps ln2),
// gamma = g/(eps ln2), c = C/(eps ln2)):
//     phi_i   <- log2 alpha_i - log2 sum_j 2^(gamma_j - c_ij)
//     gamma_j <- log2 beta_j  - log2 sum_i 2^(phi_i   - c_ij)
// from gamma = 0 (q = 1), until the row L1 error of the state after a column
// update is <= tol.  Marginals are normalised to unit mass.
//
// Absorption: each sum is evaluated around the previous potential, i.e. the
// row pass computes e_ij = 2^(phi_i + gamma_j - c_ij) with the OLD phi, whose
// row sum S_i is the current row marginal (so the stopping rule is fused into
// the pass) and whose terms are <= 1 after a column update (no overflow, no
// running max).  The first sweep, and any row whose sum leaves [1e-30, 1e30]
// (far warm starts), uses an explicit max shift instead.
//
// Fused single-read sweep (stored cost, Ncol <= 4096, Ncol % 4 == 0): a block
// owns a contiguous row range.  Bands of R rows are copied into shared memory
// by bulk asynchronous copies (TMA 1D, mbarrier completion): once for the whole
// solve when the block's rows fit ("resident", e.g. the 1024 x 1024 folded
// cost), else streamed through two stages so the next band is in flight while
// the current one is computed.  After a band's row sums give phi_new, the
// column contributions of the same entries are u_i * e_ij with u_i = alpha_i/S_i
// -- the row pass's exponentials reused, since
// 2^(phi_new_i + gamma_j - c_ij) = e_ij * alpha_i / S_i.  One cost read and ONE
// exp2 per entry per sweep.  Per-block column partials go to the workspace;
// after a grid barrier the column owners reduce them (compensated FP32 per
// warp, FP64 across warps, fixed order) and update gamma; a second barrier
// publishes gamma.
//
// Two-pass sweep (wide, odd-sized or on-the-fly costs): a row pass then a
// column pass over the cost (two exp2 per entry, no partials); the column pass
// hands out 32-column chunks through an atomic work queue.
//
// Potentials are carried in FP64 (a few values per row/column per sweep) and
// split into an FP32 hi part plus an FP32 factor 2^lo for the inner loops,
// which are pure FP32: an FP32 potential alone would bias every plan row by up
// to ulp(phi)/2 relative, above a 1e-6 marginal target when |f|/eps ~ 100.
// Each block keeps the potentials of the rows (and, in the fused kernel, the
// columns) it owns in shared memory; global copies exist only to share column
// potentials between blocks, for the rare column fallback and for the output.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace cyc {

int device_sms();

struct SkArgs {
    int M, Ncol;
    long long ld;                 // row stride of C (floats)
    const float* C;               // stored cost [M][ld] or null
    const float2* X;              // on-the-fly cost: rows' points [M]
    const float2* Y;              // columns' points [Ncol]
    const float* a;
    const float* b;
    float kappa;                  // 1 / (eps ln 2)
    double unit;                  // eps ln 2 (log2 units -> cost units)
    int stop_l2;           // 1: stop on the L2 row error (scaled by l2_scale) instead of the L1
    double l2_scale;       // 1/N for the reduced problem (its row error at the paper's scale)
    double tol;
    int max_iter;
    int check_every;
    unsigned long long timeout_ns;
    int warm;
    int debug_flags;
    double f_shift;               // added to f on output
    double* f_out;
    double* g_out;
    ot_result* res;
    // workspace
    Ctrl* ctrl;
    double* phi;                  // [2][M]  log2-unit row potentials (two buffers)
    float* fhi;                   // [2][M]  fl(phi)
    float* frf;                   // [2][M]  2^(phi - fhi)
    double* gam;                  // [2][Ncol]  log2-unit column potentials (two buffers)
    float* gc;                    // [2][Ncol]  fl(gamma)
    float* cf;                    // [2][Ncol]  2^(gamma - gc)
    float* part;                  // [grid][pstride] column partials (fused kernel)
    double* l1part;               // [grid]
    unsigned* queue;              // [2] column-chunk queue counters (two-pass kernel)
    double* acc;                  // [3][vstride] column sums + L1 (bulk-reduce kernel)
    int vstride;
    unsigned long long* trace;    // [OT_TRACE_SWEEPS][8] phase timestamps, or null
    int pstride;
    int resident;                 // fused kernel: all of a block's rows stay in shared memory
    int rows_max;                 // max rows owned by a block
    int cols_max;                 // max columns owned by a block (fused kernel)
};

// Buffers: the state after s iterations lives in buffer s & 1 (phi, gamma).
// Sweep t reads state t-1 and writes state t.

#define OT_TRACE_SWEEPS 256
__device__ __forceinline__ void trace_mark(const SkArgs& A, int t, int slot) {
    if (A.trace != nullptr && blockIdx.x == 0 && threadIdx.x == 0 && t < OT_TRACE_SWEEPS)
        A.trace[t * 8 + slot] = globaltimer();
}

__device__ __forceinline__ bool sum_ok(float s) { return s > 1e-30f && s < 1e30f; }

// Shared-memory state of the rows a block owns (dynamic shared memory).
struct RowState {
    double* phi;    // [2][rows_max]
    float* fhi;     // [2][rows_max]
    float* frf;     // [2][rows_max]
    float* alpha;   // [rows_max]
};

// ---------------------------------------------------------------------------
// shared pieces
// ---------------------------------------------------------------------------

// Marginal sums (FP64, identical order in every block) and positivity check.
__device__ bool prologue_sums(const SkArgs& A, double& inv_sa, double& inv_sb, double* s_dred) {
    double sa = 0.0, sb = 0.0;
    int bad = 0;
    for (int i = threadIdx.x; i < A.M; i += OT_BLOCK) {
        const float v = A.a[i];
        bad |= !(v > 0.f && v < INFINITY);
        sa += v;
    }
    for (int j = threadIdx.x; j < A.Ncol; j += OT_BLOCK) {
        const float v = A.b[j];
        bad |= !(v > 0.f && v < INFINITY);
        sb += v;
    }
    sa = block_sum_d(sa, s_dred);
    sb = block_sum_d(sb, s_dred);
    bad = __syncthreads_or(bad);
    inv_sa = 1.0 / sa;
    inv_sb = 1.0 / sb;
    return bad == 0;
}

__device__ __forceinline__ void store_col(const SkArgs& A, int buf, int j, double g) {
    const float hi = (float)g;
    A.gam[buf * A.Ncol + j] = g;
    A.gc[buf * A.Ncol + j] = hi;
    A.cf[buf * A.Ncol + j] = ex2((float)(g - (double)hi));
}

// Row potential for row i (local index li): shared state plus the global copy.
__device__ __forceinline__ void store_row(const SkArgs& A, const RowState& S, int buf, int i, int li, double p) {
    const float hi = (float)p;
    const float rf = ex2((float)(p - (double)hi));
    S.phi[buf * A.rows_max + li] = p;
    S.fhi[buf * A.rows_max + li] = hi;
    S.frf[buf * A.rows_max + li] = rf;
    A.phi[buf * A.M + i] = p;
    A.fhi[buf * A.M + i] = hi;
    A.frf[buf * A.M + i] = rf;
}

// Solver variant codes reported in ot_result.reserved[1].
#define OT_VARIANT_BULK 1.0
#define OT_VARIANT_FUSED 2.0
#define OT_VARIANT_TWOPASS 3.0
#define OT_VARIANT_RING 7.0

__device__ void write_result(const SkArgs& A, int iters, int status, double l1, double variant) {
    if (threadIdx.x == 0) {
        A.res->iters = iters;
        A.res->status = status;
        A.res->marg_l1 = l1;
        A.res->marg_l2_col = -1.0;
        A.res->value = 0.0;
        A.res->transport_cost = 0.0;
        A.res->marg_l1_col = -1.0;
        A.res->reserved[0] = 0.0;
        A.res->reserved[1] = variant;
    }
}

__device__ void fail_exit(const SkArgs& A) {
    if (threadIdx.x == 0) {
        A.res->iters = -1;
        A.res->status = ld_volatile_int(&A.ctrl->status);
    }
}

// Row-error term of one row (d = row sum of the current state - alpha_i, unit-mass scale):
// |d| for the L1 rule, d^2 for the L2 rule.
__device__ __forceinline__ double row_err_term(const SkArgs& A, float d) {
    return A.stop_l2 ? (double)d * (double)d : fabs((double)d);
}

// The stopping norm from the accumulated terms: the full-scale row L1, or the
// L2 row error at the paper's scale (sqrt of the sum of squares times l2_scale).
__device__ __forceinline__ double stop_norm(const SkArgs& A, double acc) {
    return A.stop_l2 ? sqrt(acc) * A.l2_scale : acc;
}

// Stopping rule on the state after `done` iterations; returns the status or -1 to continue.
__device__ __forceinline__ int stop_status(const SkArgs& A, int done, double L1) {
    if (done < 1) return -1;
    L1 = stop_norm(A, L1);
    if (L1 != L1) return OT_ERR_NONFINITE;
    if (done % A.check_every == 0 && L1 <= A.tol) return OT_OK;
    if (done >= A.max_iter) return OT_ERR_NOT_CONVERGED;
    return -1;
}

// Robust column update with an explicit max shift over the whole column, from
// the new row potentials (global buffer nb).  Whole block, one column.
// Returns the new gamma (thread 0) or NaN after recording OT_ERR_NONFINITE.
template <bool OTF>
__device__ double column_fallback(const SkArgs& A, int j, int nb, double inv_sb, float* s_redf) {
    float mx = -INFINITY;
    const float* fh = A.fhi + nb * A.M;
    const float* fr = A.frf + nb * A.M;
    for (int i = threadIdx.x; i < A.M; i += OT_BLOCK) {
        float c;
        if (OTF) {
            const float2 xi = A.X[i], yj = A.Y[j];
            const float dx = xi.x - yj.x, dy = xi.y - yj.y;
            c = fmaf(dx, dx, dy * dy);
        } else {
            c = A.C[(long long)i * A.ld + j];
        }
        mx = fmaxf(mx, fmaf(c, -A.kappa, fh[i]));
    }
    mx = warp_max(mx);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_redf[threadIdx.x >> 5] = mx;
    __syncthreads();
    float m2 = s_redf[0];
    for (int w = 1; w < OT_WARPS; ++w) m2 = fmaxf(m2, s_redf[w]);
    __syncthreads();
    float s = 0.f;
    for (int i = threadIdx.x; i < A.M; i += OT_BLOCK) {
        float c;
        if (OTF) {
            const float2 xi = A.X[i], yj = A.Y[j];
            const float dx = xi.x - yj.x, dy = xi.y - yj.y;
            c = fmaf(dx, dx, dy * dy);
        } else {
            c = A.C[(long long)i * A.ld + j];
        }
        s += ex2(fmaf(c, -A.kappa, fh[i]) - m2) * fr[i];
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) s_redf[threadIdx.x >> 5] = s;
    __syncthreads();
    double gnew = __longlong_as_double(0x7ff8000000000000ll);
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int w = 0; w < OT_WARPS; ++w) tot += s_redf[w];
        const double beta = (double)A.b[j] * inv_sb;
        if (!(tot > 0.f) || !(m2 > -INFINITY)) {
            set_status(A.ctrl, OT_ERR_NONFINITE);
        } else {
            // gamma_new = log2 beta - (m2 + log2 tot)
            gnew = (double)lg2((float)beta) - (double)m2 - (double)lg2(tot);
            store_col(A, nb, j, gnew);
        }
    }
    __syncthreads();
    return gnew;
}

// Compensated (Kahan) FP32 accumulation.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// ---------------------------------------------------------------------------
// Fused single-read kernel (stored cost, Ncol <= OT_BLOCK * CPT, Ncol % 4 == 0)
// ---------------------------------------------------------------------------

// Sum (or max) of R per-lane values over the 32 lanes of a warp, for all R at
// once: a transposing butterfly.  At offsets 16, 8, ... each lane keeps half of
// its values (the upper half if its lane bit is set) and adds the partner's
// other half; after log2(R) steps one value per lane remains, then plain xor
// steps finish the reduction.  Lane l ends with the total of value index
// (l >> (5 - log2 R)) & (R - 1).  R - 1 + (5 - log2 R) shuffles instead of 5R.
template <int R, bool MAX>
__device__ __forceinline__ float warp_reduce_rows(float (&v)[R], int lane) {
    static_assert(R == 4 || R == 8 || R == 16 || R == 32, "R must be a power of two in [4, 32]");
    constexpr int LOGR = (R == 4) ? 2 : (R == 8) ? 3 : (R == 16) ? 4 : 5;
#pragma unroll
    for (int step = 0; step < LOGR; ++step) {
        const int o = 16 >> step;
        const int half = R >> (step + 1);
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float keep = up ? v[i + half] : v[i];
            const float send = up ? v[i] : v[i + half];
            const float got = __shfl_xor_sync(0xffffffffu, send, o);
            v[i] = MAX ? fmaxf(keep, got) : keep + got;
        }
    }
    float x = v[0];
#pragma unroll
    for (int o = (16 >> LOGR); o > 0; o >>= 1) {
        const float got = __shfl_xor_sync(0xffffffffu, x, o);
        x = MAX ? fmaxf(x, got) : x + got;
    }
    return x;
}

// Band of up to R rows held in shared memory at `sb` (row stride Ncol floats).
// Thread t owns columns 4*(t + OT_BLOCK*q) + v, v < 4.  Rows r >= nr are
// computed on -inf exponents (zero entries) so that no per-row branch splits
// the work.
//
// One __syncthreads per band (two in SAFE mode): each warp reduces its R row
// partial sums with the transposing butterfly and leaves them in s_red (the
// caller alternates two buffers between bands, so a band's reads never race
// the next band's writes); after the barrier EVERY warp forms the R row sums
// lane-parallel (lane r < R sums the OT_WARPS partials of row r) and
// broadcasts the factors u_r = alpha_r / S_r by shuffles.  Lanes r < nr of
// warp 0 also record the row's L1 term (into l1, a warp-0 register) and its
// new potential, off the other warps' critical path.  On return u[] holds the
// factors; the result says whether some row sum left the safe range (the same
// answer in every thread of the block).
template <int CPT, int R, bool SAFE>
__device__ __forceinline__ bool fused_band(const SkArgs& A, const RowState& RS, const float* sb, int rb, int lb,
                                           int nr, int cur, int nxt, const float (&gcr)[CPT],
                                           const float (&cfr)[CPT], float (&e)[R][CPT], float (&u)[R], double& l1,
                                           float (*s_red)[OT_WARPS]) {
    static_assert(R <= 32, "one lane per row");
    constexpr int NV = CPT / 4;
    constexpr int LOGR = (R == 4) ? 2 : (R == 8) ? 3 : (R == 16) ? 4 : 5;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int rm = A.rows_max;
    const int my_row = (lane >> (5 - LOGR)) & (R - 1);          // row reduced into this lane
    const bool writer = (lane & ((32 >> LOGR) - 1)) == 0;        // one writer lane per row
    // 1. exponents x = gamma_j - c_ij (+ phi_i when not SAFE)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool rv = r < nr;
        const float4* srow = reinterpret_cast<const float4*>(sb + (size_t)(rv ? r : 0) * A.Ncol);
        const float F = (SAFE || !rv) ? 0.f : RS.fhi[cur * rm + lb + r];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const int g4 = tid + q * OT_BLOCK;
            if (rv && 4 * g4 < A.Ncol) {
                const float4 c = srow[g4];
                e[r][4 * q + 0] = fmaf(c.x, -A.kappa, gcr[4 * q + 0]) + F;
                e[r][4 * q + 1] = fmaf(c.y, -A.kappa, gcr[4 * q + 1]) + F;
                e[r][4 * q + 2] = fmaf(c.z, -A.kappa, gcr[4 * q + 2]) + F;
                e[r][4 * q + 3] = fmaf(c.w, -A.kappa, gcr[4 * q + 3]) + F;
            } else {
                e[r][4 * q + 0] = e[r][4 * q + 1] = e[r][4 * q + 2] = e[r][4 * q + 3] = -INFINITY;
            }
        }
    }
    float Fsafe = 0.f;   // lane r: -max of row r (SAFE)
    if (SAFE) {
        float mx[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            mx[r] = e[r][0];
#pragma unroll
            for (int q = 1; q < CPT; ++q) mx[r] = fmaxf(mx[r], e[r][q]);
        }
        const float m = warp_reduce_rows<R, true>(mx, lane);
        if (writer) s_red[my_row][wid] = m;
        __syncthreads();
        float mm = -INFINITY;
        if (lane < nr) {
#pragma unroll
            for (int w = 0; w < OT_WARPS; ++w) mm = fmaxf(mm, s_red[lane][w]);
        }
        Fsafe = (mm > -INFINITY) ? -mm : 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float F = __shfl_sync(0xffffffffu, Fsafe, r);
#pragma unroll
            for (int q = 0; q < CPT; ++q) e[r][q] += F;
        }
        __syncthreads();   // s_red is reused for the sums below
    }
    // 2. e = 2^x * colfactor, row partial sums
    float ps[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            e[r][q] = ex2(e[r][q]) * cfr[q];
            s += e[r][q];
        }
        ps[r] = s;
    }
    const float wsum = warp_reduce_rows<R, false>(ps, lane);
    if (writer) s_red[my_row][wid] = wsum;
    __syncthreads();
    // 3. every warp: lane r forms S_r, u_r; broadcast by shuffles
    float S = 1.f, alpha = 0.f;
    if (lane < nr) {
        const float4* rr = reinterpret_cast<const float4*>(s_red[lane]);
        const float4 p0 = rr[0], p1 = rr[1];
        S = ((p0.x + p0.y) + (p0.z + p0.w)) + ((p1.x + p1.y) + (p1.z + p1.w));
        alpha = RS.alpha[lb + lane];
    }
    const bool ok = (lane >= nr) || sum_ok(S);
    const float ul = (lane < nr) ? __fdividef(alpha, S) : 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) u[r] = __shfl_sync(0xffffffffu, ul, r);
    const bool bad = !__all_sync(0xffffffffu, ok);
    if (wid == 0 && lane < nr) {
        const int li = lb + lane;
        const float ratio = __fdividef(S, alpha);
        double pnew;
        if (!SAFE) {
            // L1 term of the current state: |S * 2^lo - alpha|
            l1 += row_err_term(A, fmaf(S, RS.frf[cur * rm + li] - 1.0f, S - alpha));
            pnew = (double)RS.fhi[cur * rm + li] - (double)lg2(ratio);
        } else {
            pnew = (double)Fsafe - (double)lg2(ratio);
        }
        if (ok) store_row(A, RS, nxt, rb + lane, li, pnew);
    }
    return bad;
}

// Copy band `b` of this block's rows into stage `st` (thread 0 only).
__device__ __forceinline__ void issue_band(const SkArgs& A, float* smem_bands, unsigned long long* bars, int st,
                                           int r_beg, int r_end, int R, int b) {
    const int rb = r_beg + b * R;
    const int nr = min(R, r_end - rb);
    const unsigned bytes = (unsigned)nr * (unsigned)A.Ncol * 4u;
    float* dst = smem_bands + (size_t)st * R * A.Ncol;
    mbar_arrive_expect_tx(&bars[st], bytes);
    bulk_g2s(dst, A.C + (long long)rb * A.ld, bytes, &bars[st]);
}

#define OT_MAX_STAGES 32

// Dynamic shared memory of the fused kernel: [bands][row state][column state].
__host__ __device__ inline size_t fused_rowstate_bytes(int rows_max) {
    return (size_t)rows_max * (2 * 8 + 2 * 4 + 2 * 4 + 4);
}
__host__ __device__ inline size_t fused_colstate_bytes(int cols_max) { return (size_t)cols_max * (2 * 8 + 4); }
__host__ __device__ inline size_t align256_hd(size_t x) { return (x + 255) & ~(size_t)255; }

template <int CPT, int R>
__global__ void __launch_bounds__(OT_BLOCK, 1) sk_fused_kernel(SkArgs A, int nstage_alloc) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) unsigned long long s_bar[OT_MAX_STAGES];
    __shared__ __align__(16) float s_red[2][R][OT_WARPS];
    __shared__ double s_dred[OT_WARPS];
    __shared__ float s_redf[OT_WARPS];
    __shared__ double s_colred[OT_WARPS][32];
    __shared__ int s_flag[32];
    __shared__ int s_copy_ok;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int B = blockIdx.x, G = gridDim.x;
    const int r_beg = (int)((long long)A.M * B / G), r_end = (int)((long long)A.M * (B + 1) / G);
    const int c_beg = (int)((long long)A.Ncol * B / G), c_end = (int)((long long)A.Ncol * (B + 1) / G);
    const int nbands = (r_end - r_beg + R - 1) / R;
    const bool resident = A.resident != 0;
    const int nstage = resident ? nbands : 2;

    float* smem_bands = reinterpret_cast<float*>(dsm);
    unsigned char* p = dsm + (size_t)nstage_alloc * R * A.Ncol * sizeof(float);
    RowState RS;
    RS.phi = reinterpret_cast<double*>(p);
    RS.fhi = reinterpret_cast<float*>(p + (size_t)A.rows_max * 16);
    RS.frf = RS.fhi + 2 * A.rows_max;
    RS.alpha = RS.frf + 2 * A.rows_max;
    p += align256_hd(fused_rowstate_bytes(A.rows_max));
    double* s_gam = reinterpret_cast<double*>(p);                      // [2][cols_max]
    float* s_beta = reinterpret_cast<float*>(p + (size_t)A.cols_max * 16);
    unsigned epoch = 0;

    // ---- stage the first bands (resident: all of them, once)
    if (tid == 0) {
        for (int st = 0; st < nstage; ++st) mbar_init(&s_bar[st], 1);
        fence_mbar_init();
        s_copy_ok = 1;
        if (nbands > 0) {
            const int first = resident ? nbands : min(2, nbands);
            for (int u = 0; u < first; ++u) issue_band(A, smem_bands, s_bar, u, r_beg, r_end, R, u % nbands);
        }
    }
    long long issued = nbands > 0 ? (resident ? nbands : min(2, nbands)) : 0;
    long long consumed = 0;

    double inv_sa, inv_sb;
    const bool args_ok = prologue_sums(A, inv_sa, inv_sb, s_dred);
    for (int li = tid; li < r_end - r_beg; li += OT_BLOCK) RS.alpha[li] = (float)((double)A.a[r_beg + li] * inv_sa);
    for (int j = c_beg + tid; j < c_end; j += OT_BLOCK) {
        const double g0 = A.warm ? A.g_out[j] / A.unit : 0.0;
        s_gam[j - c_beg] = g0;
        s_beta[j - c_beg] = (float)((double)A.b[j] * inv_sb);
        store_col(A, 0, j, g0);
    }
    bool go = args_ok;
    if (go && (A.debug_flags & OT_DEBUG_WITHHOLD_ARRIVAL) && B == 0) {
        withhold_arrival(A.ctrl, A.timeout_ns);
        go = false;
    } else if (go) {
        go = grid_sync(A.ctrl, G, A.timeout_ns, epoch);
    }

    for (int t = 1; go; ++t) {
        const int cur = (t - 1) & 1, nxt = cur ^ 1;
        trace_mark(A, t, 0);
        float gcr[CPT], cfr[CPT], acc[CPT];
#pragma unroll
        for (int q = 0; q < CPT / 4; ++q) {
            const int j4 = tid + q * OT_BLOCK;
            if (4 * j4 < A.Ncol) {
                const float4 g4 = reinterpret_cast<const float4*>(A.gc + cur * A.Ncol)[j4];
                const float4 c4 = reinterpret_cast<const float4*>(A.cf + cur * A.Ncol)[j4];
                gcr[4 * q] = g4.x; gcr[4 * q + 1] = g4.y; gcr[4 * q + 2] = g4.z; gcr[4 * q + 3] = g4.w;
                cfr[4 * q] = c4.x; cfr[4 * q + 1] = c4.y; cfr[4 * q + 2] = c4.z; cfr[4 * q + 3] = c4.w;
            } else {
#pragma unroll
                for (int v = 0; v < 4; ++v) { gcr[4 * q + v] = 0.f; cfr[4 * q + v] = 0.f; }
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[4 * q + v] = 0.f;
        }
        double l1 = 0.0;
        float e[R][CPT];
        for (int b = 0; b < nbands; ++b) {
            const int rb = r_beg + b * R;
            const int lb = b * R;
            const int nr = min(R, r_end - rb);
            const int st = resident ? b : (int)(consumed & 1);
            // wait for the band's copy (resident: only the first sweep)
            if (!resident || t == 1) {
                const unsigned parity = resident ? 0u : (unsigned)((consumed >> 1) & 1);
                if (tid == 0 && !mbar_wait(&s_bar[st], parity, A.timeout_ns)) {
                    set_status(A.ctrl, OT_ERR_TIMEOUT);
                    s_copy_ok = 0;
                }
                __syncthreads();
                if (!s_copy_ok) { go = false; break; }
            }
            const float* sb = smem_bands + (size_t)st * R * A.Ncol;
            float u[R];
            bool bad;
            if (t == 1) bad = fused_band<CPT, R, true>(A, RS, sb, rb, lb, nr, cur, nxt, gcr, cfr, e, u, l1, s_red[b & 1]);
            else bad = fused_band<CPT, R, false>(A, RS, sb, rb, lb, nr, cur, nxt, gcr, cfr, e, u, l1, s_red[b & 1]);
            if (bad) {   // uniform over the block: redo the band with an explicit max shift
                __syncthreads();
                double dummy = 0.0;
                if (fused_band<CPT, R, true>(A, RS, sb, rb, lb, nr, cur, nxt, gcr, cfr, e, u, dummy, s_red[b & 1]))
                    if (tid == 0) set_status(A.ctrl, OT_ERR_NONFINITE);
                __syncthreads();
            }
            // every thread has passed the band's barrier, so its shared-memory reads are
            // done: refill this stage with the band two uses ahead (streaming only)
            if (!resident) {
                ++consumed;
                if (tid == 0) {
                    fence_proxy_async();
                    issue_band(A, smem_bands, s_bar, (int)(issued & 1), r_beg, r_end, R, (int)(issued % nbands));
                }
                ++issued;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < nr) {
#pragma unroll
                    for (int q = 0; q < CPT; ++q) acc[q] = fmaf(u[r], e[r][q], acc[q]);
                }
            }
        }
        if (!go) break;
        trace_mark(A, t, 4);
#pragma unroll
        for (int q = 0; q < CPT / 4; ++q) {
            const int j4 = tid + q * OT_BLOCK;
            if (4 * j4 < A.Ncol)
                reinterpret_cast<float4*>(A.part + (long long)B * A.pstride)[j4] =
                    make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
        // only warp 0 holds L1 terms (one lane per row)
        if (wid == 0) {
            l1 = warp_sum(l1);
            if (lane == 0) A.l1part[B] = l1;
        }
        trace_mark(A, t, 1);
        if (!grid_sync(A.ctrl, G, A.timeout_ns, epoch)) { go = false; break; }
        trace_mark(A, t, 2);

        // ---- column phase: lane <-> owned column, warps split the block partials
        double l1v = 0.0;
        for (int b2 = tid; b2 < G; b2 += OT_BLOCK) l1v += ((volatile double*)A.l1part)[b2];
        for (int c0 = c_beg; c0 < c_end; c0 += 32) {
            const int j = c0 + lane;
            const bool jv = j < c_end;
            float s = 0.f, comp = 0.f;
            for (int base = 0; base < G; base += OT_WARPS * 20) {
                float v[20];   // all loads in flight before the compensated sum
#pragma unroll
                for (int k = 0; k < 20; ++k) {
                    const int b2 = base + wid + k * OT_WARPS;
                    v[k] = (jv && b2 < G) ? A.part[(long long)b2 * A.pstride + j] : 0.f;
                }
#pragma unroll
                for (int k = 0; k < 20; ++k) kahan_add(s, comp, v[k]);
            }
            s_colred[wid][lane] = (double)s - (double)comp;
            __syncthreads();
            if (wid == 0) {
                int bad = 0;
                if (jv) {
                    double R2 = 0.0;
#pragma unroll
                    for (int w = 0; w < OT_WARPS; ++w) R2 += s_colred[w][lane];
                    const int cl = j - c_beg;
                    if (R2 != R2) {
                        set_status(A.ctrl, OT_ERR_NONFINITE);
                    } else if (R2 > 1e-30 && R2 < 1e30) {
                        const double gnew = s_gam[cur * A.cols_max + cl] - (double)lg2(__fdividef((float)R2, s_beta[cl]));
                        s_gam[nxt * A.cols_max + cl] = gnew;
                        store_col(A, nxt, j, gnew);
                    } else {
                        bad = 1;
                    }
                }
                s_flag[lane] = bad;
            }
            __syncthreads();
            for (int l = 0; l < 32; ++l) {
                if (s_flag[l]) {   // rare: a column sum out of range, redo with an explicit max
                    const double gnew = column_fallback<false>(A, c0 + l, nxt, inv_sb, s_redf);
                    if (tid == 0) s_gam[nxt * A.cols_max + (c0 + l - c_beg)] = gnew;
                }
            }
        }
        trace_mark(A, t, 6);
        // ---- stopping rule on the state after iteration t-1 (its L1 was loaded above)
        const double L1 = block_sum_d(l1v, s_dred);
        trace_mark(A, t, 7);
        const int stt = stop_status(A, t - 1, L1);
        if (stt >= 0) {
            for (int li = tid; li < r_end - r_beg; li += OT_BLOCK)
                A.f_out[r_beg + li] = RS.phi[cur * A.rows_max + li] * A.unit + A.f_shift;
            for (int j = c_beg + tid; j < c_end; j += OT_BLOCK)
                A.g_out[j] = s_gam[cur * A.cols_max + (j - c_beg)] * A.unit;
            if (B == 0) write_result(A, t - 1, stt, stop_norm(A, L1), OT_VARIANT_FUSED);
            break;
        }
        trace_mark(A, t, 3);
        if (!grid_sync(A.ctrl, G, A.timeout_ns, epoch)) { go = false; break; }
    }
    if (!args_ok) {
        if (B == 0) write_result(A, 0, OT_ERR_ARG, -1.0, OT_VARIANT_FUSED);
    } else if (!go) {
        fail_exit(A);
    }
    // drain copies still in flight into this block's shared memory before leaving
    if (tid == 0 && nbands > 0) {
        if (!resident) {
            for (long long u = consumed; u < issued; ++u)
                if (!mbar_wait(&s_bar[u & 1], (unsigned)((u >> 1) & 1), A.timeout_ns)) break;
        } else {
            for (int st = 0; st < nstage; ++st) mbar_wait(&s_bar[st], 0u, A.timeout_ns);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Bulk-reduce kernel: the fused sweep with ONE grid barrier per sweep
// ---------------------------------------------------------------------------
//
// After its row phase every block adds its column partials (FP64, plus its L1
// term in slot Ncol) into one global vector with a single bulk asynchronous
// reduce-add (cp.reduce.async.bulk ... .add.f64: the TMA unit performs the
// adds at L2).  One grid barrier; then EVERY block reads the finished vector
// and updates the potentials of the columns it holds in registers (identical
// arithmetic in every block, hence identical results).  Column potentials
// never travel through global memory and there is no second barrier.  The
// vector is triple-buffered: written in sweep t, read after barrier t, zeroed
// (in slices, by all blocks) between barriers t+1 and t+2, written again in
// sweep t+3.  Each buffer may hold OT_ACC_COPIES copies (block b adds into copy
// b mod OT_ACC_COPIES, readers sum the copies); measured on GB300, one copy is
// fastest overall: spreading the L2 adds over copies shortens the barrier wait
// but costs as much again in reads.  Column potentials are FP32 hi/lo pairs
// (double-float).  FP64
// adds in a run-dependent order make the last bits of a column sum vary from
// run to run; every block still sees the same value.

// (hi, lo) -= d, renormalised (two-sum, then fast two-sum).
__device__ __forceinline__ void df_sub(float& hi, float& lo, float d) {
    const float s = hi - d;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (-d - bb);
    const float t = err + lo;
    hi = s + t;
    lo = t - (hi - s);
}

#define OT_ACC_COPIES 1

__device__ __forceinline__ void bulk_reduce_add_f64(double* gdst, const double* ssrc, unsigned bytes) {
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;" ::"l"(gdst),
                 "r"(smem_addr(ssrc)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

template <int CPT, int R>
__global__ void __launch_bounds__(OT_BLOCK, 1) sk_bulk_kernel(SkArgs A, int nstage_alloc) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) unsigned long long s_bar[OT_MAX_STAGES];
    __shared__ __align__(16) float s_red[2][R][OT_WARPS];
    __shared__ double s_dred[OT_WARPS];
    __shared__ float s_redf[OT_WARPS];
    __shared__ int s_copy_ok;
    __shared__ int s_nfix;
    __shared__ int s_fix[64];

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int B = blockIdx.x, G = gridDim.x;
    const int Nc = A.Ncol;
    const int vlen = Nc + 2;                     // column sums, L1, pad
    const int r_beg = (int)((long long)A.M * B / G), r_end = (int)((long long)A.M * (B + 1) / G);
    const int o_beg = (int)((long long)Nc * B / G), o_end = (int)((long long)Nc * (B + 1) / G);
    const long long zlen = (long long)OT_ACC_COPIES * A.vstride;   // one buffer, all copies
    const int z_beg = (int)(zlen * B / G), z_end = (int)(zlen * (B + 1) / G);
    const int nbands = (r_end - r_beg + R - 1) / R;
    const bool resident = A.resident != 0;
    const int nstage = resident ? nbands : 2;

    float* smem_bands = reinterpret_cast<float*>(dsm);
    unsigned char* p = dsm + (size_t)nstage_alloc * R * Nc * sizeof(float);
    double* s_part = reinterpret_cast<double*>(p);                     // [vlen]
    p += align256_hd((size_t)vlen * sizeof(double));
    float* s_glo = reinterpret_cast<float*>(p);                        // [Ncol] gamma lo
    float* s_ghi = s_glo + Nc;                                         // [Ncol] gamma hi
    float* s_beta = s_ghi + Nc;                                        // [Ncol]
    p += align256_hd((size_t)3 * Nc * sizeof(float));
    RowState RS;
    RS.phi = reinterpret_cast<double*>(p);
    RS.fhi = reinterpret_cast<float*>(p + (size_t)A.rows_max * 16);
    RS.frf = RS.fhi + 2 * A.rows_max;
    RS.alpha = RS.frf + 2 * A.rows_max;
    double* acc_g = A.acc;                                              // [3][vstride]
    unsigned epoch = 0;

    if (tid == 0) {
        for (int st = 0; st < nstage; ++st) mbar_init(&s_bar[st], 1);
        fence_mbar_init();
        s_copy_ok = 1;
        s_nfix = 0;
        if (nbands > 0) {
            const int first = resident ? nbands : min(2, nbands);
            for (int u = 0; u < first; ++u) issue_band(A, smem_bands, s_bar, u, r_beg, r_end, R, u % nbands);
        }
    }
    long long issued = nbands > 0 ? (resident ? nbands : min(2, nbands)) : 0;
    long long consumed = 0;

    double inv_sa, inv_sb;
    const bool args_ok = prologue_sums(A, inv_sa, inv_sb, s_dred);
    for (int li = tid; li < r_end - r_beg; li += OT_BLOCK) RS.alpha[li] = (float)((double)A.a[r_beg + li] * inv_sa);
    for (int j = tid; j < Nc; j += OT_BLOCK) s_beta[j] = (float)((double)A.b[j] * inv_sb);
    float gcr[CPT], cfr[CPT];
#pragma unroll
    for (int q = 0; q < CPT / 4; ++q) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int j = 4 * (tid + q * OT_BLOCK) + v;
            float hi = 0.f, lo = 0.f;
            if (j < Nc) {
                const double g0 = A.warm ? A.g_out[j] / A.unit : 0.0;
                split_f64(g0, hi, lo);
                s_ghi[j] = hi;
                s_glo[j] = lo;
            }
            gcr[4 * q + v] = hi;
            cfr[4 * q + v] = (j < Nc) ? ex2(lo) : 0.f;
        }
    }
    bool go = args_ok;
    if (go && (A.debug_flags & OT_DEBUG_WITHHOLD_ARRIVAL) && B == 0) {
        withhold_arrival(A.ctrl, A.timeout_ns);
        go = false;
    } else if (go) {
        go = grid_sync(A.ctrl, G, A.timeout_ns, epoch);
    }

    for (int t = 1; go; ++t) {
        const int cur = (t - 1) & 1, nxt = cur ^ 1;
        const size_t bufsz = (size_t)OT_ACC_COPIES * A.vstride;
        double* vec = acc_g + (size_t)(t % 3) * bufsz;                  // this sweep's sums (all copies)
        double* vmine = vec + (size_t)(B % OT_ACC_COPIES) * A.vstride;  // the copy this block adds into
        double* vzero = acc_g + (size_t)((t + 2) % 3) * bufsz;          // read in sweep t-1: clear it
        trace_mark(A, t, 0);
        float acc[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[q] = 0.f;
        double l1 = 0.0;
        float e[R][CPT];
        for (int b = 0; b < nbands; ++b) {
            const int rb = r_beg + b * R;
            const int lb = b * R;
            const int nr = min(R, r_end - rb);
            const int st = resident ? b : (int)(consumed & 1);
            if (!resident || t == 1) {
                const unsigned parity = resident ? 0u : (unsigned)((consumed >> 1) & 1);
                if (tid == 0 && !mbar_wait(&s_bar[st], parity, A.timeout_ns)) {
                    set_status(A.ctrl, OT_ERR_TIMEOUT);
                    s_copy_ok = 0;
                }
                __syncthreads();
                if (!s_copy_ok) { go = false; break; }
            }
            const float* sb = smem_bands + (size_t)st * R * Nc;
            float u[R];
            bool bad;
            if (t == 1) bad = fused_band<CPT, R, true>(A, RS, sb, rb, lb, nr, cur, nxt, gcr, cfr, e, u, l1, s_red[b & 1]);
            else bad = fused_band<CPT, R, false>(A, RS, sb, rb, lb, nr, cur, nxt, gcr, cfr, e, u, l1, s_red[b & 1]);
            if (bad) {   // uniform over the block: redo the band with an explicit max shift
                __syncthreads();
                double dummy = 0.0;
                if (fused_band<CPT, R, true>(A, RS, sb, rb, lb, nr, cur, nxt, gcr, cfr, e, u, dummy, s_red[b & 1]))
                    if (tid == 0) set_status(A.ctrl, OT_ERR_NONFINITE);
                __syncthreads();
            }
            if (!resident) {
                ++consumed;
                if (tid == 0) {
                    fence_proxy_async();
                    issue_band(A, smem_bands, s_bar, (int)(issued & 1), r_beg, r_end, R, (int)(issued % nbands));
                }
                ++issued;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < nr) {
#pragma unroll
                    for (int q = 0; q < CPT; ++q) acc[q] = fmaf(u[r], e[r][q], acc[q]);
                }
            }
        }
        if (!go) break;
        trace_mark(A, t, 4);
        // ---- block partials (FP64) + L1 into shared memory, one bulk reduce-add into the global vector
#pragma unroll
        for (int q = 0; q < CPT / 4; ++q) {
            const int j4 = tid + q * OT_BLOCK;
            if (4 * j4 < Nc) {
                double2* dst = reinterpret_cast<double2*>(s_part + 4 * j4);
                dst[0] = make_double2((double)acc[4 * q], (double)acc[4 * q + 1]);
                dst[1] = make_double2((double)acc[4 * q + 2], (double)acc[4 * q + 3]);
            }
        }
        if (wid == 0) {   // only warp 0 holds L1 terms (one lane per row)
            l1 = warp_sum(l1);
            if (lane == 0) { s_part[Nc] = l1; s_part[Nc + 1] = 0.0; }
        }
        fence_proxy_async();   // this thread's shared-memory writes -> visible to the bulk copy
        __syncthreads();
        if (tid == 0) {
            fence_proxy_async_global();   // the slice clears of earlier sweeps precede this reduce
            // two pieces starting at a block-dependent offset (a multiple of 2 doubles), so the
            // blocks' adds do not all hit the same L2 sectors at the same time
            const int rot = (int)(((long long)(vlen / 2) * B / G) * 2);
            if (rot > 0) bulk_reduce_add_f64(vmine, s_part, (unsigned)(rot * sizeof(double)));
            bulk_reduce_add_f64(vmine + rot, s_part + rot, (unsigned)((vlen - rot) * sizeof(double)));
            bulk_wait_all();
            fence_proxy_async_global();
        }
        trace_mark(A, t, 1);
        if (!grid_sync(A.ctrl, G, A.timeout_ns, epoch)) { go = false; break; }
        trace_mark(A, t, 2);

        // ---- column sums of this thread's columns and the L1 of the state, all loads issued
        // before any use: every copy's entries unconditionally (clamped index), L1 lane-parallel
        double2 r01[CPT / 4][OT_ACC_COPIES], r23[CPT / 4][OT_ACC_COPIES];
#pragma unroll
        for (int q = 0; q < CPT / 4; ++q) {
            const int j4 = min(tid + q * OT_BLOCK, Nc / 4 - 1);
#pragma unroll
            for (int c = 0; c < OT_ACC_COPIES; ++c) {
                const double2* src = reinterpret_cast<const double2*>(vec + (size_t)c * A.vstride + 4 * j4);
                r01[q][c] = __ldcg(src);
                r23[q][c] = __ldcg(src + 1);
            }
        }
        double L1 = (lane < OT_ACC_COPIES) ? __ldcg(vec + (size_t)lane * A.vstride + Nc) : 0.0;
        L1 = warp_sum(L1);
        double Rcol[CPT];
#pragma unroll
        for (int q = 0; q < CPT / 4; ++q) {
            // pairwise sums of the copies (fixed order)
#pragma unroll
            for (int w = OT_ACC_COPIES / 2; w > 0; w /= 2)
#pragma unroll
                for (int c = 0; c < w; ++c) {
                    r01[q][c].x += r01[q][c + w].x; r01[q][c].y += r01[q][c + w].y;
                    r23[q][c].x += r23[q][c + w].x; r23[q][c].y += r23[q][c + w].y;
                }
            Rcol[4 * q] = r01[q][0].x; Rcol[4 * q + 1] = r01[q][0].y;
            Rcol[4 * q + 2] = r23[q][0].x; Rcol[4 * q + 3] = r23[q][0].y;
        }
        trace_mark(A, t, 5);
        const int stt = stop_status(A, t - 1, L1);
        if (stt >= 0) {
            for (int li = tid; li < r_end - r_beg; li += OT_BLOCK)
                A.f_out[r_beg + li] = RS.phi[cur * A.rows_max + li] * A.unit + A.f_shift;
            for (int j = o_beg + tid; j < o_end; j += OT_BLOCK)
                A.g_out[j] = ((double)s_ghi[j] + (double)s_glo[j]) * A.unit;
            if (B == 0) write_result(A, t - 1, stt, stop_norm(A, L1), OT_VARIANT_BULK);
            break;
        }
#pragma unroll
        for (int q = 0; q < CPT / 4; ++q) {
            const int j4 = tid + q * OT_BLOCK;
            if (4 * j4 < Nc) {
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int j = 4 * j4 + v;
                    const double Rj = Rcol[4 * q + v];
                    if (Rj != Rj) {
                        set_status(A.ctrl, OT_ERR_NONFINITE);
                    } else if (Rj > 1e-30 && Rj < 1e30) {
                        float hi = gcr[4 * q + v], lo = s_glo[j];
                        df_sub(hi, lo, lg2(__fdividef((float)Rj, s_beta[j])));
                        gcr[4 * q + v] = hi;
                        cfr[4 * q + v] = ex2(lo);
                        s_ghi[j] = hi;
                        s_glo[j] = lo;
                    } else {
                        const int k2 = atomicAdd(&s_nfix, 1);
                        if (k2 < 64) s_fix[k2] = j;
                        else set_status(A.ctrl, OT_ERR_NONFINITE);
                    }
                }
            }
        }
        trace_mark(A, t, 6);
        // clear this block's slice of the vector read in sweep t-1 (next written in sweep t+2)
        if (z_beg + tid < z_end) {
            for (int k = z_beg + tid; k < z_end; k += OT_BLOCK) vzero[k] = 0.0;   // slice of all copies
            fence_proxy_async_global();   // by the writing threads: clears ordered before later bulk adds
        }
        __syncthreads();
        trace_mark(A, t, 7);
        const int nfix = min(s_nfix, 64);
        if (nfix > 0) {   // rare: column sums out of range, recomputed with an explicit max by every block
            for (int k = 0; k < nfix; ++k) {
                const int j = s_fix[k];
                const double gnew = column_fallback<false>(A, j, nxt, inv_sb, s_redf);
                if (tid == 0) {
                    float hi, lo;
                    split_f64(gnew, hi, lo);
                    s_ghi[j] = hi;
                    s_glo[j] = lo;
                }
            }
            __syncthreads();
            if (tid == 0) s_nfix = 0;
#pragma unroll
            for (int q = 0; q < CPT / 4; ++q)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int j = 4 * (tid + q * OT_BLOCK) + v;
                    if (j < Nc) { gcr[4 * q + v] = s_ghi[j]; cfr[4 * q + v] = ex2(s_glo[j]); }
                }
            __syncthreads();
        }
        trace_mark(A, t, 3);
    }
    if (!args_ok) {
        if (B == 0) write_result(A, 0, OT_ERR_ARG, -1.0, OT_VARIANT_BULK);
    } else if (!go) {
        fail_exit(A);
    }
    if (tid == 0 && nbands > 0) {
        if (!resident) {
            for (long long u = consumed; u < issued; ++u)
                if (!mbar_wait(&s_bar[u & 1], (unsigned)((u >> 1) & 1), A.timeout_ns)) break;
        } else {
            for (int st = 0; st < nstage; ++st) mbar_wait(&s_bar[st], 0u, A.timeout_ns);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Ring kernel: per-thread asynchronous-copy ring, FP32 sweep, one grid barrier
// ---------------------------------------------------------------------------
//
// The same single-read sweep as the kernels above (one cost read and one exp2
// per entry, row sums around the previous row potential, column contributions
// u_i * e_ij from the row pass's exponentials), laid out for 512 threads:
//
// * Cost bands reach shared memory by per-thread 16-byte asynchronous copies
//   (cp.async.cg, L2 only): each thread copies exactly the float4 slots it
//   later reads, so a band needs no block barrier to become visible -- each
//   thread waits for its own copy groups (cp.async.wait_group).  S stages are
//   in flight per block; a stage is refilled as soon as its thread has turned
//   the band's costs into exponentials.  The ring runs across sweeps (the next
//   sweep's first bands load during the column exchange).  When all of a
//   block's rows fit, they are copied once and stay resident.
// * Every arithmetic step of a sweep is FP32 (this GPU's FP64 pipe, and its
//   FP32 <-> FP64 conversions, are far slower than FP32): potentials are
//   (hi, lo) pairs updated by error-free transformations, and the column
//   partials are converted to FP64 bit patterns by integer operations.
// * The column sums are added at L2 in FP64 by one bulk reduce-add per block
//   (cp.reduce.async.bulk .add.f64) into a triple-buffered vector, followed by
//   ONE grid barrier; then every block reads the vector and updates the
//   potentials of all columns in registers (identical arithmetic everywhere).

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// x >= 0 (FP32) -> the same value as an FP64 bit pattern, by integer operations:
// exact for normal x; zero and the flush-to-zero range give 0, Inf and NaN give NaN.
__device__ __forceinline__ double f32_to_f64_bits(float x) {
    const unsigned b = __float_as_uint(x) & 0x7fffffffu;
    const unsigned e = b >> 23;
    unsigned long long d = ((unsigned long long)b << 29) + (896ull << 52);
    d = (e == 0u) ? 0ull : d;
    d = (e == 255u) ? 0x7ff8000000000000ull : d;
    return __longlong_as_double((long long)d);
}

// x >= 0 (FP64) -> nearest FP32 (ties away from zero) by integer operations; below the
// FP32 normal range -> 0, above -> Inf, Inf and NaN -> NaN.
__device__ __forceinline__ float f64_to_f32_bits(double x) {
    const unsigned long long d = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    const unsigned e = (unsigned)(d >> 52);
    const unsigned r = (unsigned)((d - (896ull << 52) + (1ull << 28)) >> 29);
    float f = __uint_as_float(r);
    f = (e < 897u) ? 0.f : f;
    f = (e > 1150u) ? __uint_as_float(0x7f800000u) : f;
    f = (e == 0x7ffu) ? __uint_as_float(0x7fc00000u) : f;
    return f;
}

// (hi, lo) = a - d exactly (two-difference).
__device__ __forceinline__ void two_diff(float a, float d, float& hi, float& lo) {
    const float s = a - d;
    const float bb = s - a;
    lo = (a - (s - bb)) + (-d - bb);
    hi = s;
}

// Shared-memory row state of the ring kernel (rows the block owns).
struct RingRows {
    float* hi;      // [2][rows_max]  hi part of the row potential (log2 units)
    float* lo;      // [2][rows_max]  lo part
    float* fr;      // [2][rows_max]  2^lo
    float* alpha;   // [rows_max]     normalised row marginal
};

// Issue the copies of band `band` of this block into ring stage `st` (this thread's slots).
template <int NT, int CPT, int R>
__device__ __forceinline__ void ring_issue(const SkArgs& A, float* ring, int st, int r_beg, int r_end, int band) {
    const int rb = r_beg + band * R;
    const int nr = min(R, r_end - rb);
    float* dst = ring + (size_t)st * R * A.Ncol;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r < nr) {
#pragma unroll
            for (int q = 0; q < CPT / 4; ++q) {
                const int j4 = threadIdx.x + q * NT;
                if (4 * j4 < A.Ncol) cp_async16(dst + (size_t)r * A.Ncol + 4 * j4, A.C + (long long)(rb + r) * A.ld + 4 * j4);
            }
        }
    }
}

// One band of up to R rows, from ring stage `sb` (row stride rstride floats) or, with
// GSRC, straight from the cost rows in global memory.  Exponents from the thread's own
// slots, exp2, row sums (one block barrier), factors u_r = alpha_r / S_r for every
// thread, new row potentials and the row L1 terms (warp 0).  The callback `refill`
// runs once the stage's contents are in registers.  Returns true when some row sum
// left the safe range (the same answer in every thread).
template <int NT, int CPT, int R, bool SAFE, bool GSRC, typename Refill>
__device__ __forceinline__ bool ring_band(const SkArgs& A, const RingRows& RS, const float* sb, long long rstride,
                                          int rb, int lb, int nr,
                                          int cur, int nxt, const float (&ghi)[CPT], const float (&cf)[CPT],
                                          float (&e)[R][CPT], float (&u)[R], float& l1, float (*s_red)[NT / 32],
                                          Refill refill) {
    constexpr int NW = NT / 32;
    constexpr int NV = CPT / 4;
    constexpr int LOGR = (R == 4) ? 2 : (R == 8) ? 3 : (R == 16) ? 4 : 5;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int rm = A.rows_max;
    const int my_row = (lane >> (5 - LOGR)) & (R - 1);
    const bool writer = (lane & ((32 >> LOGR) - 1)) == 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool rv = r < nr;
        const float F = (SAFE || !rv) ? 0.f : RS.hi[cur * rm + lb + r];
        const float4* srow = reinterpret_cast<const float4*>(sb + (rv ? r : 0) * rstride);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const int j4 = tid + q * NT;
            if (rv && 4 * j4 < A.Ncol) {
                const float4 c = GSRC ? __ldg(srow + j4) : srow[j4];
                e[r][4 * q + 0] = fmaf(c.x, -A.kappa, ghi[4 * q + 0]) + F;
                e[r][4 * q + 1] = fmaf(c.y, -A.kappa, ghi[4 * q + 1]) + F;
                e[r][4 * q + 2] = fmaf(c.z, -A.kappa, ghi[4 * q + 2]) + F;
                e[r][4 * q + 3] = fmaf(c.w, -A.kappa, ghi[4 * q + 3]) + F;
            } else {
                e[r][4 * q + 0] = e[r][4 * q + 1] = e[r][4 * q + 2] = e[r][4 * q + 3] = -INFINITY;
            }
        }
    }
    refill();   // the stage's costs now live in registers
    float Fsafe = 0.f;
    if (SAFE) {
        float mx[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            mx[r] = e[r][0];
#pragma unroll
            for (int q = 1; q < CPT; ++q) mx[r] = fmaxf(mx[r], e[r][q]);
        }
        const float m = warp_reduce_rows<R, true>(mx, lane);
        if (writer) s_red[my_row][wid] = m;
        __syncthreads();
        float mm = -INFINITY;
        if (lane < nr) {
#pragma unroll
            for (int w = 0; w < NW; ++w) mm = fmaxf(mm, s_red[lane][w]);
        }
        Fsafe = (mm > -INFINITY) ? -mm : 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float F = __shfl_sync(0xffffffffu, Fsafe, r);
#pragma unroll
            for (int q = 0; q < CPT; ++q) e[r][q] += F;
        }
        __syncthreads();   // s_red is reused for the sums below
    }
    float ps[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            e[r][q] = ex2(e[r][q]);
            s = fmaf(e[r][q], cf[q], s);
        }
        ps[r] = s;
    }
    const float wsum = warp_reduce_rows<R, false>(ps, lane);
    if (writer) s_red[my_row][wid] = wsum;
    __syncthreads();
    float S = 1.f, alpha = 0.f;
    if (lane < nr) {
        const float4* rr = reinterpret_cast<const float4*>(s_red[lane]);
        float4 acc4 = rr[0];
#pragma unroll
        for (int w = 1; w < NW / 4; ++w) {
            const float4 p = rr[w];
            acc4.x += p.x; acc4.y += p.y; acc4.z += p.z; acc4.w += p.w;
        }
        S = (acc4.x + acc4.y) + (acc4.z + acc4.w);
        alpha = RS.alpha[lb + lane];
    }
    const bool ok = (lane >= nr) || sum_ok(S);
    const float ul = (lane < nr) ? __fdividef(alpha, S) : 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) u[r] = __shfl_sync(0xffffffffu, ul, r);
    const bool bad = !__all_sync(0xffffffffu, ok);
    if (wid == 0 && lane < nr) {
        const int li = lb + lane;
        const float d = lg2(__fdividef(S, alpha));
        float base;
        if (!SAFE) {
            // L1 term of the current state: |S * 2^lo - alpha|; a row out of range counts as unconverged
            l1 += ok ? fabsf(fmaf(S, RS.fr[cur * rm + li] - 1.0f, S - alpha)) : 1e30f;
            base = RS.hi[cur * rm + li];
        } else {
            base = Fsafe;
        }
        if (ok) {
            float h, l;
            two_diff(base, d, h, l);
            const float f = ex2(l);
            RS.hi[nxt * rm + li] = h;
            RS.lo[nxt * rm + li] = l;
            RS.fr[nxt * rm + li] = f;
            A.fhi[nxt * A.M + rb + lane] = h;
            A.frf[nxt * A.M + rb + lane] = f;
        }
    }
    return bad;
}

// Column potential from scratch with an explicit max shift over the column (rare: the
// column sum left the safe range).  Whole block; every thread gets (hi, lo).
template <int NT>
__device__ void ring_column_fallback(const SkArgs& A, int j, int nb, float beta, float* s_redf, float& hi,
                                     float& lo) {
    constexpr int NW = NT / 32;
    const float* fh = A.fhi + nb * A.M;
    const float* fr = A.frf + nb * A.M;
    float mx = -INFINITY;
    for (int i = threadIdx.x; i < A.M; i += NT) mx = fmaxf(mx, fmaf(A.C[(long long)i * A.ld + j], -A.kappa, fh[i]));
    mx = warp_max(mx);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_redf[threadIdx.x >> 5] = mx;
    __syncthreads();
    float m2 = s_redf[0];
    for (int w = 1; w < NW; ++w) m2 = fmaxf(m2, s_redf[w]);
    __syncthreads();
    float s = 0.f;
    for (int i = threadIdx.x; i < A.M; i += NT) s += ex2(fmaf(A.C[(long long)i * A.ld + j], -A.kappa, fh[i]) - m2) * fr[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) s_redf[threadIdx.x >> 5] = s;
    __syncthreads();
    float tot = 0.f;
    for (int w = 0; w < NW; ++w) tot += s_redf[w];
    __syncthreads();
    if (!(tot > 0.f) || !(m2 > -INFINITY) || !(beta > 0.f)) {
        if (threadIdx.x == 0) set_status(A.ctrl, OT_ERR_NONFINITE);
        hi = 0.f;
        lo = 0.f;
        return;
    }
    // gamma = log2 beta - m2 - log2 tot
    two_diff(lg2(beta), m2, hi, lo);
    df_sub(hi, lo, lg2(tot));
}

template <int NT, int CPT, int R, int S>
__global__ void __launch_bounds__(NT, 1) sk_ring_kernel(SkArgs A) {
    constexpr int NW = NT / 32;
    constexpr int NV = CPT / 4;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(16) float s_red[2][R][NW];
    __shared__ float s_redf[NW];
    __shared__ int s_nfix;
    __shared__ int s_fix[64];
    __shared__ float s_fixv[64][2];

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int B = blockIdx.x, G = gridDim.x;
    const int Nc = A.Ncol;
    const int r_beg = (int)((long long)A.M * B / G), r_end = (int)((long long)A.M * (B + 1) / G);
    const int o_beg = (int)((long long)Nc * B / G), o_end = (int)((long long)Nc * (B + 1) / G);
    const int z_beg = (int)((long long)A.vstride * B / G), z_end = (int)((long long)A.vstride * (B + 1) / G);
    const int nbands = (r_end - r_beg + R - 1) / R;
    const bool resident = A.resident != 0;
    const int lsl = NV * 4 * NT;   // the L1 slot of the column-sum vector

    // dynamic shared memory: [ring][partials (4 NT + 2 doubles)][row state]
    float* ring = reinterpret_cast<float*>(dsm);
    const int nstage = resident ? nbands : S;
    unsigned char* p = dsm + align256_hd((size_t)nstage * R * Nc * sizeof(float));
    double* s_part = reinterpret_cast<double*>(p);
    p += align256_hd((size_t)(4 * NT + 2) * sizeof(double));
    RingRows RS;
    RS.hi = reinterpret_cast<float*>(p);
    RS.lo = RS.hi + 2 * A.rows_max;
    RS.fr = RS.lo + 2 * A.rows_max;
    RS.alpha = RS.fr + 2 * A.rows_max;
    unsigned epoch = 0;

    // ---- first copies: every band (resident) or the first S bands of the ring
    int ref_band = 0;   // band the next refill copies (wrapping)
    if (nbands > 0) {
        if (resident) {
            for (int b = 0; b < nbands; ++b) ring_issue<NT, CPT, R>(A, ring, b, r_beg, r_end, b);
            cp_async_commit();
        } else {
            for (int s = 0; s < S; ++s) {
                ring_issue<NT, CPT, R>(A, ring, s, r_beg, r_end, s % nbands);
                cp_async_commit();
            }
            ref_band = S % nbands;
        }
    }
    int st_next = 0;    // stage read next (wrapping)

    __shared__ double s_dred[NW];
    double sa = 0.0, sb = 0.0;   // marginal sums (FP64, once per solve)
    int badm = 0;
    for (int i = tid; i < A.M; i += NT) { const float v = A.a[i]; badm |= !(v > 0.f && v < INFINITY); sa += v; }
    for (int j = tid; j < Nc; j += NT) { const float v = A.b[j]; badm |= !(v > 0.f && v < INFINITY); sb += v; }
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    if (lane == 0) s_dred[wid] = sa;
    __syncthreads();
    double tsa = 0.0;
    for (int w = 0; w < NW; ++w) tsa += s_dred[w];
    __syncthreads();
    if (lane == 0) s_dred[wid] = sb;
    __syncthreads();
    double tsb = 0.0;
    for (int w = 0; w < NW; ++w) tsb += s_dred[w];
    const bool args_ok = __syncthreads_or(badm) == 0;
    const double inv_sa = 1.0 / tsa, inv_sb = 1.0 / tsb;
    for (int li = tid; li < r_end - r_beg; li += NT) RS.alpha[li] = (float)((double)A.a[r_beg + li] * inv_sa);
    if (tid == 0) s_nfix = 0;
    // column state in registers: potentials (hi, lo), 2^lo, normalised column marginal
    float ghi[CPT], glo[CPT], cf[CPT], beta[CPT];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int j = 4 * (tid + q * NT) + v;
            float hi = 0.f, lo = 0.f, bt = 1.f;
            if (j < Nc) {
                const double g0 = A.warm ? A.g_out[j] / A.unit : 0.0;
                split_f64(g0, hi, lo);
                bt = (float)((double)A.b[j] * inv_sb);
            }
            ghi[4 * q + v] = hi;
            glo[4 * q + v] = lo;
            cf[4 * q + v] = (j < Nc) ? ex2(lo) : 0.f;
            beta[4 * q + v] = bt;
        }
    }
    const float tolf = (float)A.tol;
    bool go = args_ok;
    if (go && (A.debug_flags & OT_DEBUG_WITHHOLD_ARRIVAL) && B == 0) {
        withhold_arrival(A.ctrl, A.timeout_ns);
        go = false;
    } else if (go) {
        go = grid_sync(A.ctrl, G, A.timeout_ns, epoch);
    }

    for (int t = 1; go; ++t) {
        const int cur = (t - 1) & 1, nxt = cur ^ 1;
        double* vec = A.acc + (size_t)(t % 3) * A.vstride;
        double* vzero = A.acc + (size_t)((t + 2) % 3) * A.vstride;
        trace_mark(A, t, 0);
        float acc[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[q] = 0.f;
        float l1 = 0.f;
        float e[R][CPT];
        if (resident && t == 1) cp_async_wait_all();
        for (int b = 0; b < nbands; ++b) {
            const int rb = r_beg + b * R;
            const int lb = b * R;
            const int nr = min(R, r_end - rb);
            int st = b;
            if (!resident) {
                cp_async_wait<S - 1>();
                st = st_next;
                st_next = (st_next + 1 == S) ? 0 : st_next + 1;
            }
            const float* sbase = ring + (size_t)st * R * Nc;
            auto refill = [&]() {
                if (!resident) {
                    ring_issue<NT, CPT, R>(A, ring, st, r_beg, r_end, ref_band);
                    cp_async_commit();
                    ref_band = (ref_band + 1 == nbands) ? 0 : ref_band + 1;
                }
            };
            auto none = []() {};
            float u[R];
            bool bad;
            if (t == 1)
                bad = ring_band<NT, CPT, R, true, false>(A, RS, sbase, Nc, rb, lb, nr, cur, nxt, ghi, cf, e, u, l1,
                                                         s_red[b & 1], refill);
            else
                bad = ring_band<NT, CPT, R, false, false>(A, RS, sbase, Nc, rb, lb, nr, cur, nxt, ghi, cf, e, u, l1,
                                                          s_red[b & 1], refill);
            if (bad) {   // uniform over the block: redo the band max-shifted, its costs re-read from global memory
                __syncthreads();   // (the ring stage may already hold the next band)
                float dummy = 0.f;
                if (ring_band<NT, CPT, R, true, true>(A, RS, A.C + (long long)rb * A.ld, A.ld, rb, lb, nr, cur, nxt, ghi,
                                                      cf, e, u, dummy, s_red[b & 1], none))
                    if (tid == 0) set_status(A.ctrl, OT_ERR_NONFINITE);
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < nr) {
#pragma unroll
                    for (int q = 0; q < CPT; ++q) acc[q] = fmaf(u[r], e[r][q], acc[q]);
                }
            }
        }
        trace_mark(A, t, 4);
        // ---- column partials (FP64 bit patterns) and the L1 term: one bulk reduce-add per chunk of 4 NT columns
        if (wid == 0) l1 = warp_sum(l1);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            if (q > 0) {
                if (tid == 0) bulk_wait_read();   // the previous chunk has left shared memory
                __syncthreads();
            }
            double2* dst = reinterpret_cast<double2*>(s_part + 4 * tid);
            dst[0] = make_double2(f32_to_f64_bits(acc[4 * q]), f32_to_f64_bits(acc[4 * q + 1]));
            dst[1] = make_double2(f32_to_f64_bits(acc[4 * q + 2]), f32_to_f64_bits(acc[4 * q + 3]));
            const bool last = q == NV - 1;
            if (last && tid == 0) {
                s_part[4 * NT] = f32_to_f64_bits(l1);
                s_part[4 * NT + 1] = 0.0;
            }
            fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                if (q == 0) fence_proxy_async_global();   // the slice clears of earlier sweeps precede these adds
                bulk_reduce_add_f64(vec + 4 * NT * q, s_part, (unsigned)((4 * NT + (last ? 2 : 0)) * sizeof(double)));
            }
        }
        if (tid == 0) {
            bulk_wait_all();
            fence_proxy_async_global();
        }
        trace_mark(A, t, 1);
        if (!grid_sync(A.ctrl, G, A.timeout_ns, epoch)) { go = false; break; }
        trace_mark(A, t, 2);

        // ---- column sums of this thread's columns and the L1 of the state after t - 1 iterations
        double2 v01[NV], v23[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const double2* src = reinterpret_cast<const double2*>(vec + 4 * (tid + q * NT));
            v01[q] = __ldcg(src);
            v23[q] = __ldcg(src + 1);
        }
        const double L1d = __ldcg(vec + lsl);
        const float L1 = f64_to_f32_bits(L1d);
        trace_mark(A, t, 5);
        int stt = -1;
        if (t - 1 >= 1) {
            if (L1 != L1) stt = OT_ERR_NONFINITE;
            else if ((t - 1) % A.check_every == 0 && L1 <= tolf) stt = OT_OK;
            else if (t - 1 >= A.max_iter) stt = OT_ERR_NOT_CONVERGED;
        }
        if (stt >= 0) {
            for (int li = tid; li < r_end - r_beg; li += NT)
                A.f_out[r_beg + li] =
                    ((double)RS.hi[cur * A.rows_max + li] + (double)RS.lo[cur * A.rows_max + li]) * A.unit + A.f_shift;
#pragma unroll
            for (int q = 0; q < NV; ++q)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int j = 4 * (tid + q * NT) + v;
                    if (j >= o_beg && j < o_end) A.g_out[j] = ((double)ghi[4 * q + v] + (double)glo[4 * q + v]) * A.unit;
                }
            if (B == 0 && tid == 0) {
                A.res->iters = t - 1;
                A.res->status = stt;
                A.res->marg_l1 = L1d;
                A.res->marg_l2_col = -1.0;
                A.res->value = 0.0;
                A.res->transport_cost = 0.0;
                A.res->marg_l1_col = -1.0;
                A.res->reserved[0] = 0.0;
                A.res->reserved[1] = OT_VARIANT_RING;
            }
            break;
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const float Av[4] = {f64_to_f32_bits(v01[q].x), f64_to_f32_bits(v01[q].y), f64_to_f32_bits(v23[q].x),
                                 f64_to_f32_bits(v23[q].y)};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int k = 4 * q + v;
                const int j = 4 * (tid + q * NT) + v;
                if (j < Nc) {
                    const float Rj = Av[v] * cf[k];   // column sum of the plan after the row update
                    if (Rj != Rj) {
                        set_status(A.ctrl, OT_ERR_NONFINITE);
                    } else if (Rj > 1e-30f && Rj < 1e30f) {
                        df_sub(ghi[k], glo[k], lg2(__fdividef(Rj, beta[k])));
                        cf[k] = ex2(glo[k]);
                    } else {
                        const int k2 = atomicAdd(&s_nfix, 1);
                        if (k2 < 64) s_fix[k2] = j;
                        else set_status(A.ctrl, OT_ERR_NONFINITE);
                    }
                }
            }
        }
        trace_mark(A, t, 6);
        // clear this block's slice of the vector read in sweep t-1 (next written in sweep t+2)
        if (z_beg + tid < z_end) {
            for (int k = z_beg + tid; k < z_end; k += NT) vzero[k] = 0.0;
            fence_proxy_async_global();
        }
        __syncthreads();
        const int nfix = min(s_nfix, 64);
        if (nfix > 0) {   // rare: column sums out of range, recomputed with an explicit max by every block
            for (int k = 0; k < nfix; ++k) {
                const int j = s_fix[k];
                float h, l;
                ring_column_fallback<NT>(A, j, nxt, (float)((double)A.b[j] * inv_sb), s_redf, h, l);
                if (tid == 0) { s_fixv[k][0] = h; s_fixv[k][1] = l; }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < NV; ++q)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int j = 4 * (tid + q * NT) + v;
                    for (int k = 0; k < nfix; ++k)
                        if (s_fix[k] == j) {
                            ghi[4 * q + v] = s_fixv[k][0];
                            glo[4 * q + v] = s_fixv[k][1];
                            cf[4 * q + v] = ex2(s_fixv[k][1]);
                        }
                }
            __syncthreads();
            if (tid == 0) s_nfix = 0;
            __syncthreads();
        }
        trace_mark(A, t, 3);
    }
    if (!args_ok) {
        if (B == 0 && tid == 0) {
            A.res->iters = 0;
            A.res->status = OT_ERR_ARG;
            A.res->marg_l1 = -1.0;
            A.res->reserved[1] = OT_VARIANT_RING;
        }
    } else if (!go) {
        fail_exit(A);
    }
    cp_async_wait_all();   // no copy may still target this block's shared memory when it exits
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Ping-pong ring kernel: two independent warp groups, owner-reduced columns
// ---------------------------------------------------------------------------
//
// The ring kernel's sweep with the block split into two groups of 256 threads
// that take alternate bands of the block's rows.  Each group synchronises on
// its own named barrier only, so one group's row reduction overlaps the other
// group's exponentials.  Both groups hold every column of the block
// (thread t of a group owns columns 4 (t + 256 q) + v), and their column
// partials are added in shared memory at the end of the row phase.
//
// Column exchange (no FP64 and no atomics: deterministic): every block stores
// its FP32 column partials and row-error term; grid barrier; block B reduces
// the ~m/G columns it owns over all blocks' partials (compensated FP32, fixed
// order), updates their potentials and publishes them as (hi, lo) pairs;
// grid barrier; every thread reads the potentials of its columns.  The row-
// error terms are summed in the same fixed order in every block, so every
// block takes the same stopping decision.

#define PP_G 256   // threads per group

typedef unsigned long long pf2;   // two packed FP32 values (f32x2 instructions)
__device__ __forceinline__ pf2 p2(float a, float b) {
    pf2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 u2(pf2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return make_float2(a, b);
}
__device__ __forceinline__ pf2 fma_p2(pf2 a, pf2 b, pf2 c) {
    pf2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ pf2 add_p2(pf2 a, pf2 b) {
    pf2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ pf2 ex2_p2(pf2 x) {
    const float2 v = u2(x);
    return p2(ex2(v.x), ex2(v.y));
}

__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(PP_G) : "memory");
}

// Sum of R per-lane values over a warp for all R at once (R = 2: one transposing
// step, then plain xor steps).  Lane l ends with the total of value (l >> 4) & 1.
template <int R>
__device__ __forceinline__ float warp_reduce_rows2(float (&v)[R], int lane) {
    if constexpr (R == 2) {
        const bool up = (lane & 16) != 0;
        const float keep = up ? v[1] : v[0];
        const float send = up ? v[0] : v[1];
        float x = keep + __shfl_xor_sync(0xffffffffu, send, 16);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        return x;
    } else {
        return warp_reduce_rows<R, false>(v, lane);
    }
}

// Copies of band `band` into stage `st` of group g (this thread's slots only).
template <int CPT, int R>
__device__ __forceinline__ void pp_issue(const SkArgs& A, float* gring, int st, int r_beg, int r_end, int band,
                                         int gt, unsigned cvalid, bool full_cols) {
    const int rb = r_beg + band * R;
    const int nr = min(R, r_end - rb);
    float* dst = gring + (size_t)st * R * A.Ncol + 4 * gt;
    const float* src = A.C + (long long)rb * A.ld + 4 * gt;
    if (nr == R && full_cols) {   // the common case: no per-slot tests
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < CPT / 4; ++q)
                cp_async16(dst + (size_t)r * A.Ncol + 4 * PP_G * q, src + (long long)r * A.ld + 4 * PP_G * q);
        return;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r < nr) {
#pragma unroll
            for (int q = 0; q < CPT / 4; ++q)
                if (cvalid & (1u << q)) cp_async16(dst + (size_t)r * A.Ncol + 4 * PP_G * q, src + (long long)r * A.ld + 4 * PP_G * q);
        }
    }
}

// One band of up to R rows for group g.  SAFE: explicit max shift (first sweep, and
// the rare redo when a row sum left the safe range); GSRC: costs from global memory.
// Returns true when some row sum left the safe range (uniform over the group).
template <int CPT, int R, bool SAFE, bool GSRC, bool FULL, typename Refill>
__device__ __forceinline__ bool pp_band(const SkArgs& A, const RingRows& RS, const float* sb, long long rstride,
                                        int rb, int lb, int nr, int cur, int nxt, int g, int gt, unsigned cvalid,
                                        const pf2 (&gh)[CPT / 2], const pf2* __restrict__ scf, pf2 (&e)[R][CPT / 2],
                                        float (&u)[R], float& l1, float (*s_red)[8], Refill refill) {
    constexpr int NV = CPT / 4;
    const int lane = gt & 31, wg = gt >> 5;
    const int rm = A.rows_max;
    const pf2 nk = p2(-A.kappa, -A.kappa);
    constexpr int LOGR = (R == 2) ? 1 : (R == 4) ? 2 : 3;
    const int my_row = (lane >> (5 - LOGR)) & (R - 1);
    const bool writer = (lane & ((32 >> LOGR) - 1)) == 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool rv = FULL || r < nr;
        const float F = (SAFE || !rv) ? 0.f : RS.hi[cur * rm + lb + r];
        const pf2 FF = p2(F, F);
        const float* srow = sb + (rv ? r : 0) * rstride + 4 * gt;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            if (FULL || (rv && (cvalid & (1u << q)))) {
                const float4 c = GSRC ? __ldg(reinterpret_cast<const float4*>(srow + 4 * PP_G * q))
                                      : *reinterpret_cast<const float4*>(srow + 4 * PP_G * q);
                e[r][2 * q] = add_p2(fma_p2(p2(c.x, c.y), nk, gh[2 * q]), FF);
                e[r][2 * q + 1] = add_p2(fma_p2(p2(c.z, c.w), nk, gh[2 * q + 1]), FF);
            } else {
                e[r][2 * q] = e[r][2 * q + 1] = p2(-INFINITY, -INFINITY);
            }
        }
    }
    refill();   // the stage's costs are in registers
    float Fsafe = 0.f;
    if (SAFE) {
        float mx[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float m = -INFINITY;
#pragma unroll
            for (int q = 0; q < CPT / 2; ++q) {
                const float2 v = u2(e[r][q]);
                m = fmaxf(m, fmaxf(v.x, v.y));
            }
            mx[r] = m;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) mx[r] = warp_max(mx[r]);
        if (lane == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) s_red[r][wg] = mx[r];
        }
        group_sync(g);
        float mm = -INFINITY;
        if (lane < nr) {
#pragma unroll
            for (int w = 0; w < 8; ++w) mm = fmaxf(mm, s_red[lane][w]);
        }
        Fsafe = (mm > -INFINITY) ? -mm : 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float F = __shfl_sync(0xffffffffu, Fsafe, r);
            const pf2 FF = p2(F, F);
#pragma unroll
            for (int q = 0; q < CPT / 2; ++q) e[r][q] = add_p2(e[r][q], FF);
        }
        group_sync(g);   // s_red is reused for the sums below
    }
    float ps[R];
    pf2 cf[CPT / 2];   // the column factors 2^lo, read from shared memory for this band only
#pragma unroll
    for (int q = 0; q < CPT / 2; ++q) cf[q] = scf[q * PP_G + gt];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        pf2 s2 = p2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < CPT / 2; ++q) {
            e[r][q] = ex2_p2(e[r][q]);
            s2 = fma_p2(e[r][q], cf[q], s2);
        }
        const float2 s = u2(s2);
        ps[r] = s.x + s.y;
    }
    const float wsum = warp_reduce_rows2<R>(ps, lane);
    if (writer) s_red[my_row][wg] = wsum;
    group_sync(g);
    float S = 1.f, alpha = 0.f;
    if (lane < nr) {
        const float4* rr = reinterpret_cast<const float4*>(s_red[lane]);
        const float4 p0 = rr[0], p1 = rr[1];
        S = ((p0.x + p0.y) + (p0.z + p0.w)) + ((p1.x + p1.y) + (p1.z + p1.w));
        alpha = RS.alpha[lb + lane];
    }
    const bool ok = (lane >= nr) || sum_ok(S);
    const float ul = (lane < nr) ? __fdividef(alpha, S) : 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) u[r] = __shfl_sync(0xffffffffu, ul, r);
    const bool bad = !__all_sync(0xffffffffu, ok);
    if (wg == 0 && lane < nr) {
        const int li = lb + lane;
        const float d = lg2(__fdividef(S, alpha));
        float base;
        if (!SAFE) {
            l1 += ok ? fabsf(fmaf(S, RS.fr[cur * rm + li] - 1.0f, S - alpha)) : 1e30f;
            base = RS.hi[cur * rm + li];
        } else {
            base = Fsafe;
        }
        if (ok) {
            float h, l;
            two_diff(base, d, h, l);
            const float f = ex2(l);
            RS.hi[nxt * rm + li] = h;
            RS.lo[nxt * rm + li] = l;
            RS.fr[nxt * rm + li] = f;
            A.fhi[nxt * A.M + rb + lane] = h;
            A.frf[nxt * A.M + rb + lane] = f;
        }
    }
    return bad;
}

template <int CPT, int R, int S>
__global__ void __launch_bounds__(2 * PP_G, 1) sk_pp_kernel(SkArgs A) {
    constexpr int NV = CPT / 4;
    constexpr int NT = 2 * PP_G;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(16) float s_red[2][2][R][8];   // [group][band parity][row][warp of the group]
    __shared__ float s_redf[NW];
    __shared__ float s_own[16][2][33];                  // owner phase: [slice][sum, comp][column]
    __shared__ float s_l1g[2];
    __shared__ float s_L1;
    __shared__ int s_fix;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int g = tid / PP_G, gt = tid % PP_G;
    const int B = blockIdx.x, G = gridDim.x;
    const int Nc = A.Ncol;
    const int r_beg = (int)((long long)A.M * B / G), r_end = (int)((long long)A.M * (B + 1) / G);
    const int o_beg = (int)((long long)Nc * B / G), o_end = (int)((long long)Nc * (B + 1) / G);
    const int nown = o_end - o_beg;   // <= 32 (checked by the launcher)
    const int nbands = (r_end - r_beg + R - 1) / R;
    const int gbands = (nbands - g + 1) / 2;          // bands g, g + 2, ... of this block
    const bool resident = A.resident != 0;
    const int nstage = resident ? (nbands + 1) / 2 : S;
    unsigned cvalid = 0;
#pragma unroll
    for (int q = 0; q < NV; ++q) cvalid |= (4 * (gt + PP_G * q) < Nc) ? (1u << q) : 0u;

    // dynamic shared memory: [group 0 ring][group 1 ring][group-1 column partials][row state][owned columns]
    const size_t gring_floats = (size_t)nstage * R * Nc;
    float* gring = reinterpret_cast<float*>(dsm) + (size_t)g * gring_floats;
    unsigned char* p = dsm + align256_hd(2 * gring_floats * sizeof(float));
    float* s_acc = reinterpret_cast<float*>(p);                 // [PP_G][CPT]
    p += align256_hd((size_t)PP_G * CPT * sizeof(float));
    pf2* s_cf = reinterpret_cast<pf2*>(p);                      // [CPT / 2][PP_G] column factors 2^lo
    p += align256_hd((size_t)PP_G * CPT * sizeof(float));
    RingRows RS;
    RS.hi = reinterpret_cast<float*>(p);
    RS.lo = RS.hi + 2 * A.rows_max;
    RS.fr = RS.lo + 2 * A.rows_max;
    RS.alpha = RS.fr + 2 * A.rows_max;
    p += align256_hd((size_t)A.rows_max * 7 * sizeof(float));
    float* s_ohi = reinterpret_cast<float*>(p);   // owned columns: potential (hi, lo), 2^lo, beta
    float* s_olo = s_ohi + 32;
    float* s_ocf = s_olo + 32;
    float* s_obt = s_ocf + 32;
    float2* gam2 = reinterpret_cast<float2*>(A.gc);   // [2][Ncol] published (hi, lo) per state
    unsigned epoch = 0;

    // ---- first copies of this group's bands; then the stage to consume next and the
    // band (of this group) the next refill copies, both as wrapping counters
    // every thread of the block holds only valid columns: a block-uniform condition, so the
    // fast path (which holds warp-synchronous shuffles) is taken by whole groups or not at all
    const bool full_cols = Nc == 4 * PP_G * NV;
    int st_next = 0, ref_band = 0;
    if (gbands > 0) {
        if (resident) {
            for (int bb = 0; bb < gbands; ++bb)
                pp_issue<CPT, R>(A, gring, bb, r_beg, r_end, 2 * bb + g, gt, cvalid, full_cols);
            cp_async_commit();
        } else {
            for (int s = 0; s < S; ++s) {
                pp_issue<CPT, R>(A, gring, s, r_beg, r_end, 2 * (s % gbands) + g, gt, cvalid, full_cols);
                cp_async_commit();
            }
            ref_band = S % gbands;
        }
    }

    __shared__ double s_dred[NW];
    double sa = 0.0, sb = 0.0;
    int badm = 0;
    for (int i = tid; i < A.M; i += NT) { const float v = A.a[i]; badm |= !(v > 0.f && v < INFINITY); sa += v; }
    for (int j = tid; j < Nc; j += NT) { const float v = A.b[j]; badm |= !(v > 0.f && v < INFINITY); sb += v; }
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    if (lane == 0) s_dred[wid] = sa;
    __syncthreads();
    double tsa = 0.0;
    for (int w = 0; w < NW; ++w) tsa += s_dred[w];
    __syncthreads();
    if (lane == 0) s_dred[wid] = sb;
    __syncthreads();
    double tsb = 0.0;
    for (int w = 0; w < NW; ++w) tsb += s_dred[w];
    const bool args_ok = __syncthreads_or(badm) == 0;
    const double inv_sa = 1.0 / tsa, inv_sb = 1.0 / tsb;
    for (int li = tid; li < r_end - r_beg; li += NT) RS.alpha[li] = (float)((double)A.a[r_beg + li] * inv_sa);
    // potentials of this thread's columns, and the owned columns' full state
    pf2 gh[CPT / 2];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        float hv[4], cv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int j = 4 * (gt + PP_G * q) + v;
            float hi = 0.f, lo = 0.f;
            if (j < Nc && A.warm) split_f64(A.g_out[j] / A.unit, hi, lo);
            hv[v] = hi;
            cv[v] = (j < Nc) ? ex2(lo) : 0.f;
        }
        gh[2 * q] = p2(hv[0], hv[1]);
        gh[2 * q + 1] = p2(hv[2], hv[3]);
        if (g == 0) {
            s_cf[(2 * q) * PP_G + gt] = p2(cv[0], cv[1]);
            s_cf[(2 * q + 1) * PP_G + gt] = p2(cv[2], cv[3]);
        }
    }
    if (tid < nown) {
        const int j = o_beg + tid;
        float hi = 0.f, lo = 0.f;
        if (A.warm) split_f64(A.g_out[j] / A.unit, hi, lo);
        s_ohi[tid] = hi;
        s_olo[tid] = lo;
        s_ocf[tid] = ex2(lo);
        s_obt[tid] = (float)((double)A.b[j] * inv_sb);
    }
    if (tid == 0) s_fix = 0;
    const float tolf = (float)A.tol;
    bool go = args_ok;
    if (go && (A.debug_flags & OT_DEBUG_WITHHOLD_ARRIVAL) && B == 0) {
        withhold_arrival(A.ctrl, A.timeout_ns);
        go = false;
    } else if (go) {
        go = grid_sync(A.ctrl, G, A.timeout_ns, epoch);
    }

    for (int t = 1; go; ++t) {
        const int cur = (t - 1) & 1, nxt = cur ^ 1;
        trace_mark(A, t, 0);
        pf2 acc[CPT / 2];
#pragma unroll
        for (int q = 0; q < CPT / 2; ++q) acc[q] = p2(0.f, 0.f);
        float l1 = 0.f;
        pf2 e[R][CPT / 2];
        if (resident && t == 1) cp_async_wait_all();
        for (int bb = 0; bb < gbands; ++bb) {
            const int b = 2 * bb + g;
            const int rb = r_beg + b * R;
            const int lb = b * R;
            const int nr = min(R, r_end - rb);
            int st = bb;
            if (!resident) {
                cp_async_wait<S - 1>();
                st = st_next;
                st_next = (st_next + 1 == S) ? 0 : st_next + 1;
            }
            const float* sbase = gring + (size_t)st * R * Nc;
            auto refill = [&]() {
                if (!resident) {
                    pp_issue<CPT, R>(A, gring, st, r_beg, r_end, 2 * ref_band + g, gt, cvalid, full_cols);
                    cp_async_commit();
                    ref_band = (ref_band + 1 == gbands) ? 0 : ref_band + 1;
                }
            };
            auto none = []() {};
            float u[R];
            bool bad;
            if (t == 1)
                bad = pp_band<CPT, R, true, false, false>(A, RS, sbase, Nc, rb, lb, nr, cur, nxt, g, gt, cvalid, gh, s_cf,
                                                          e, u, l1, s_red[g][bb & 1], refill);
            else if (nr == R && full_cols)
                bad = pp_band<CPT, R, false, false, true>(A, RS, sbase, Nc, rb, lb, nr, cur, nxt, g, gt, cvalid, gh, s_cf,
                                                          e, u, l1, s_red[g][bb & 1], refill);
            else
                bad = pp_band<CPT, R, false, false, false>(A, RS, sbase, Nc, rb, lb, nr, cur, nxt, g, gt, cvalid, gh,
                                                           s_cf, e, u, l1, s_red[g][bb & 1], refill);
            if (bad) {   // uniform over the group: redo the band max-shifted from the costs in global memory
                group_sync(g);
                float dummy = 0.f;
                if (pp_band<CPT, R, true, true, false>(A, RS, A.C + (long long)rb * A.ld, A.ld, rb, lb, nr, cur, nxt, g,
                                                       gt, cvalid, gh, s_cf, e, u, dummy, s_red[g][bb & 1], none))
                    if (gt == 0) set_status(A.ctrl, OT_ERR_NONFINITE);
                group_sync(g);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < nr) {
                    const pf2 uu = p2(u[r], u[r]);
#pragma unroll
                    for (int q = 0; q < CPT / 2; ++q) acc[q] = fma_p2(uu, e[r][q], acc[q]);
                }
            }
        }
        trace_mark(A, t, 4);
        // ---- the two groups' column partials and row-error terms -> one per block, to global memory
        if (wid == 0 || wid == PP_G / 32) {
            const float v = warp_sum(l1);
            if (lane == 0) s_l1g[g] = v;
        }
        if (g == 1) {
#pragma unroll
            for (int q = 0; q < CPT / 2; ++q) reinterpret_cast<pf2*>(s_acc)[q * PP_G + gt] = acc[q];
        }
        __syncthreads();
        if (g == 0) {
            float* prow = A.part + (long long)B * A.pstride;
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                if (cvalid & (1u << q)) {
                    const float2 a0 = u2(add_p2(acc[2 * q], reinterpret_cast<const pf2*>(s_acc)[(2 * q) * PP_G + gt]));
                    const float2 a1 =
                        u2(add_p2(acc[2 * q + 1], reinterpret_cast<const pf2*>(s_acc)[(2 * q + 1) * PP_G + gt]));
                    __stcg(reinterpret_cast<float4*>(prow + 4 * (gt + PP_G * q)), make_float4(a0.x, a0.y, a1.x, a1.y));
                }
            }
            if (gt == 0) reinterpret_cast<float*>(A.l1part)[B] = s_l1g[0] + s_l1g[1];
        }
        trace_mark(A, t, 1);
        if (!grid_sync(A.ctrl, G, A.timeout_ns, epoch)) { go = false; break; }
        trace_mark(A, t, 2);

        // ---- owner phase: the owned columns' sums over all blocks (compensated FP32, fixed order)
        // and the row L1 of the state after t - 1 iterations (the last warp, same order in every
        // block); every load is issued before any arithmetic
        {
            const int c = tid & 31, sl = tid >> 5;   // column of the owned range, slice of the blocks
            float v[10], lv[5];
#pragma unroll
            for (int k = 0; k < 10; ++k) {
                const int b2 = sl + 16 * k;
                v[k] = (c < nown && b2 < G) ? __ldcg(A.part + (long long)b2 * A.pstride + o_beg + c) : 0.f;
            }
            if (wid == NW - 1) {
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const int b2 = lane + 32 * k;
                    lv[k] = (b2 < G) ? __ldcg(reinterpret_cast<const float*>(A.l1part) + b2) : 0.f;
                }
            }
            float s = 0.f, cp = 0.f;
#pragma unroll
            for (int k = 0; k < 10; ++k) kahan_add(s, cp, v[k]);
            if (c < nown)
                for (int b2 = sl + 160; b2 < G; b2 += 16) kahan_add(s, cp, __ldcg(A.part + (long long)b2 * A.pstride + o_beg + c));
            s_own[sl][0][c] = s;
            s_own[sl][1][c] = cp;
            if (wid == NW - 1) {
                float ls = 0.f, lc = 0.f;
#pragma unroll
                for (int k = 0; k < 5; ++k) kahan_add(ls, lc, lv[k]);
                for (int b2 = lane + 160; b2 < G; b2 += 32) kahan_add(ls, lc, __ldcg(reinterpret_cast<const float*>(A.l1part) + b2));
                ls -= lc;
                ls = warp_sum(ls);
                if (lane == 0) s_L1 = ls;
            }
        }
        __syncthreads();
        const float L1 = s_L1;
        trace_mark(A, t, 5);
        int stt = -1;
        if (t - 1 >= 1) {
            if (L1 != L1) stt = OT_ERR_NONFINITE;
            else if ((t - 1) % A.check_every == 0 && L1 <= tolf) stt = OT_OK;
            else if (t - 1 >= A.max_iter) stt = OT_ERR_NOT_CONVERGED;
        }
        if (stt >= 0) {
            for (int li = tid; li < r_end - r_beg; li += NT)
                A.f_out[r_beg + li] =
                    ((double)RS.hi[cur * A.rows_max + li] + (double)RS.lo[cur * A.rows_max + li]) * A.unit + A.f_shift;
            if (tid < nown) A.g_out[o_beg + tid] = ((double)s_ohi[tid] + (double)s_olo[tid]) * A.unit;
            if (B == 0 && tid == 0) {
                A.res->iters = t - 1;
                A.res->status = stt;
                A.res->marg_l1 = (double)L1;
                A.res->marg_l2_col = -1.0;
                A.res->value = 0.0;
                A.res->transport_cost = 0.0;
                A.res->marg_l1_col = -1.0;
                A.res->reserved[0] = 0.0;
                A.res->reserved[1] = OT_VARIANT_RING;
            }
            break;
        }
        // half-warp h (of warps 0..15) combines the 16 slices of owned column c = h with TwoSum merges
        // (fixed tree, the same in every block), then its lane 0 updates the column's potential
        {
            const int c = tid >> 4, sl = tid & 15;
            float s = 0.f, cp = 0.f;
            if (c < nown) {
                s = s_own[sl][0][c];
                cp = s_own[sl][1][c];
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {   // (s, cp) + partner's: exact sum of the two hi parts
                const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, cp, o);
                const float t = s + s2;
                const float bb = t - s;
                const float err = (s - (t - bb)) + (s2 - bb);
                cp = cp + c2 - err;
                s = t;
            }
            if (sl == 0 && c < nown) {
                s -= cp;
                const float Rj = s * s_ocf[c];   // column sum of the plan after the row update
                if (Rj != Rj) {
                    set_status(A.ctrl, OT_ERR_NONFINITE);
                } else if (Rj > 1e-30f && Rj < 1e30f) {
                    float hi = s_ohi[c], lo = s_olo[c];
                    df_sub(hi, lo, lg2(__fdividef(Rj, s_obt[c])));
                    s_ohi[c] = hi;
                    s_olo[c] = lo;
                    s_ocf[c] = ex2(lo);
                    gam2[nxt * Nc + o_beg + c] = make_float2(hi, lo);
                } else {
                    atomicAdd(&s_fix, 1);
                    s_ohi[c] = NAN;   // marks the column for the fallback below
                }
            }
        }
        __syncthreads();
        if (s_fix > 0) {   // rare: a column sum out of range, recomputed with an explicit max over the column
            for (int c = 0; c < nown; ++c) {
                if (!(s_ohi[c] == s_ohi[c])) {
                    float h, l;
                    ring_column_fallback<NT>(A, o_beg + c, nxt, s_obt[c], s_redf, h, l);
                    if (tid == 0) {
                        s_ohi[c] = h;
                        s_olo[c] = l;
                        s_ocf[c] = ex2(l);
                        gam2[nxt * Nc + o_beg + c] = make_float2(h, l);
                    }
                    __syncthreads();
                }
            }
            if (tid == 0) s_fix = 0;
        }
        trace_mark(A, t, 6);
        if (!grid_sync(A.ctrl, G, A.timeout_ns, epoch)) { go = false; break; }
        // ---- every thread: the new potentials of its columns (every slot is redefined, so the old
        // values are not kept alive through the exchange)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            float4 h01 = make_float4(0.f, 0.f, 0.f, 0.f), h23 = h01;
            if (cvalid & (1u << q)) {
                const float4* src = reinterpret_cast<const float4*>(gam2 + nxt * Nc + 4 * (gt + PP_G * q));
                h01 = __ldcg(src);   // (hi, lo) of 4 columns
                h23 = __ldcg(src + 1);
            }
            gh[2 * q] = p2(h01.x, h01.z);
            gh[2 * q + 1] = p2(h23.x, h23.z);
            if (g == 0) {
                s_cf[(2 * q) * PP_G + gt] = p2(ex2(h01.y), ex2(h01.w));
                s_cf[(2 * q + 1) * PP_G + gt] = p2(ex2(h23.y), ex2(h23.w));
            }
        }
        __syncthreads();   // the column factors are read by both groups in the next sweep
        trace_mark(A, t, 3);
    }
    if (!args_ok) {
        if (B == 0 && tid == 0) {
            A.res->iters = 0;
            A.res->status = OT_ERR_ARG;
            A.res->marg_l1 = -1.0;
            A.res->reserved[1] = OT_VARIANT_RING;
        }
    } else if (!go) {
        fail_exit(A);
    }
    cp_async_wait_all();   // no copy may still target this block's shared memory when it exits
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Two-pass kernel (any width; stored or on-the-fly cost)
// ---------------------------------------------------------------------------

#define WR 8   // rows per band in the two-pass row phase

// Row phase for a band of up to WR rows: S_r = sum_j 2^(F_r + gamma_j - c_rj) * cf_j.
// SAFE: F_r = -max_j(gamma_j - c_rj) (extra pass).  Writes phi_new; adds L1.
template <bool OTF, bool SAFE>
__device__ void twopass_row_band(const SkArgs& A, const RowState& RS, int rb, int lb, int nr, int cur, int nxt,
                                 double& l1, float (*s_red)[WR], float* s_F, int* s_bad) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int rm = A.rows_max;
    const float* gcp = A.gc + cur * A.Ncol;
    const float* cfp = A.cf + cur * A.Ncol;
    float F[WR];
    float2 xr[WR];
    const float* crow[WR];
#pragma unroll
    for (int r = 0; r < WR; ++r) {
        const int row = rb + (r < nr ? r : 0);
        xr[r] = OTF ? __ldg(A.X + row) : make_float2(0.f, 0.f);
        crow[r] = OTF ? nullptr : A.C + (long long)row * A.ld;
        F[r] = (!SAFE && r < nr) ? RS.fhi[cur * rm + lb + r] : 0.f;
    }
    if (SAFE) {
        float mx[WR];
#pragma unroll
        for (int r = 0; r < WR; ++r) mx[r] = -INFINITY;
        for (int j = tid; j < A.Ncol; j += OT_BLOCK) {
            const float g = gcp[j];
            float2 yj = make_float2(0.f, 0.f);
            if (OTF) yj = __ldg(A.Y + j);
#pragma unroll
            for (int r = 0; r < WR; ++r) {
                if (r < nr) {
                    float c;
                    if (OTF) {
                        const float dx = xr[r].x - yj.x, dy = xr[r].y - yj.y;
                        c = fmaf(dx, dx, dy * dy);
                    } else {
                        c = __ldg(crow[r] + j);
                    }
                    mx[r] = fmaxf(mx[r], fmaf(c, -A.kappa, g));
                }
            }
        }
#pragma unroll
        for (int r = 0; r < WR; ++r) {
            const float m = warp_max(mx[r]);
            if (lane == 0) s_red[wid][r] = m;
        }
        __syncthreads();
        if (tid < WR) {
            float m = s_red[0][tid];
            for (int w = 1; w < OT_WARPS; ++w) m = fmaxf(m, s_red[w][tid]);
            s_F[tid] = (tid < nr && m > -INFINITY) ? -m : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < WR; ++r) F[r] = s_F[r];
    }
    float s[WR], sc[WR];   // compensated sums: up to n / OT_BLOCK terms per thread
#pragma unroll
    for (int r = 0; r < WR; ++r) s[r] = sc[r] = 0.f;
    for (int j = tid; j < A.Ncol; j += OT_BLOCK) {
        const float g = gcp[j], cfj = cfp[j];
        float2 yj = make_float2(0.f, 0.f);
        if (OTF) yj = __ldg(A.Y + j);
#pragma unroll
        for (int r = 0; r < WR; ++r) {
            if (r < nr) {
                float c;
                if (OTF) {
                    const float dx = xr[r].x - yj.x, dy = xr[r].y - yj.y;
                    c = fmaf(dx, dx, dy * dy);
                } else {
                    c = __ldg(crow[r] + j);
                }
                kahan_add(s[r], sc[r], ex2(fmaf(c, -A.kappa, g) + F[r]) * cfj);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < WR; ++r) {
        const float v = warp_sum(s[r] - sc[r]);
        if (lane == 0) s_red[wid][r] = v;
    }
    __syncthreads();
    if (tid < nr) {
        const int li = lb + tid;
        float S = 0.f;
        for (int w = 0; w < OT_WARPS; ++w) S += s_red[w][tid];
        const float alpha = RS.alpha[li];
        double pnew;
        if (!SAFE) {
            l1 += row_err_term(A, fmaf(S, RS.frf[cur * rm + li] - 1.0f, S - alpha));
            pnew = (double)RS.fhi[cur * rm + li] - (double)lg2(S / alpha);
        } else {
            pnew = (double)s_F[tid] - (double)lg2(S / alpha);
        }
        if (sum_ok(S)) store_row(A, RS, nxt, rb + tid, li, pnew);
        else *s_bad = 1;
    }
    __syncthreads();
}

template <bool OTF>
__global__ void __launch_bounds__(OT_BLOCK, 1) sk_twopass_kernel(SkArgs A) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ float s_red[OT_WARPS][WR];
    __shared__ float s_F[WR];
    __shared__ int s_bad;
    __shared__ double s_dred[OT_WARPS];
    __shared__ float s_redf[OT_WARPS];
    __shared__ float s_col[OT_WARPS][32];
    __shared__ int s_flag[32];
    __shared__ unsigned s_chunk;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int B = blockIdx.x, G = gridDim.x;
    const int r_beg = (int)((long long)A.M * B / G), r_end = (int)((long long)A.M * (B + 1) / G);
    // static column ranges (initialisation and output), in chunks of 32
    const int nchunks = (A.Ncol + 31) / 32;
    const int k_beg = (int)((long long)nchunks * B / G), k_end = (int)((long long)nchunks * (B + 1) / G);
    const int c_beg = min(A.Ncol, k_beg * 32), c_end = min(A.Ncol, k_end * 32);
    RowState RS;
    RS.phi = reinterpret_cast<double*>(dsm);
    RS.fhi = reinterpret_cast<float*>(dsm + (size_t)A.rows_max * 16);
    RS.frf = RS.fhi + 2 * A.rows_max;
    RS.alpha = RS.frf + 2 * A.rows_max;
    unsigned epoch = 0;

    double inv_sa, inv_sb;
    const bool args_ok = prologue_sums(A, inv_sa, inv_sb, s_dred);
    for (int li = tid; li < r_end - r_beg; li += OT_BLOCK) RS.alpha[li] = (float)((double)A.a[r_beg + li] * inv_sa);
    for (int j = c_beg + tid; j < c_end; j += OT_BLOCK) store_col(A, 0, j, A.warm ? A.g_out[j] / A.unit : 0.0);
    if (B == 0 && tid == 0) { A.queue[0] = 0; A.queue[1] = 0; }
    if (tid == 0) s_bad = 0;
    bool go = args_ok;
    if (go && (A.debug_flags & OT_DEBUG_WITHHOLD_ARRIVAL) && B == 0) {
        withhold_arrival(A.ctrl, A.timeout_ns);
        go = false;
    } else if (go) {
        go = grid_sync(A.ctrl, G, A.timeout_ns, epoch);
    }

    for (int t = 1; go; ++t) {
        const int cur = (t - 1) & 1, nxt = cur ^ 1;
        trace_mark(A, t, 0);
        double l1 = 0.0;
        for (int rb = r_beg; rb < r_end; rb += WR) {
            const int nr = min(WR, r_end - rb);
            const int lb = rb - r_beg;
            if (t == 1) twopass_row_band<OTF, true>(A, RS, rb, lb, nr, cur, nxt, l1, s_red, s_F, &s_bad);
            else twopass_row_band<OTF, false>(A, RS, rb, lb, nr, cur, nxt, l1, s_red, s_F, &s_bad);
            if (s_bad) {
                __syncthreads();
                if (tid == 0) s_bad = 0;
                double dummy = 0.0;
                twopass_row_band<OTF, true>(A, RS, rb, lb, nr, cur, nxt, dummy, s_red, s_F, &s_bad);
                if (s_bad) {
                    if (tid == 0) { set_status(A.ctrl, OT_ERR_NONFINITE); s_bad = 0; }
                    __syncthreads();
                }
            }
        }
        // only warp 0 holds L1 terms (one lane per row)
        if (wid == 0) {
            l1 = warp_sum(l1);
            if (lane == 0) A.l1part[B] = l1;
        }
        trace_mark(A, t, 1);
        if (!grid_sync(A.ctrl, G, A.timeout_ns, epoch)) { go = false; break; }
        trace_mark(A, t, 2);

        double l1v = 0.0;
        for (int b2 = tid; b2 < G; b2 += OT_BLOCK) l1v += ((volatile double*)A.l1part)[b2];
        const double L1 = block_sum_d(l1v, s_dred);
        const int stt = stop_status(A, t - 1, L1);
        if (stt >= 0) {
            for (int li = tid; li < r_end - r_beg; li += OT_BLOCK)
                A.f_out[r_beg + li] = RS.phi[cur * A.rows_max + li] * A.unit + A.f_shift;
            for (int j = c_beg + tid; j < c_end; j += OT_BLOCK) A.g_out[j] = A.gam[cur * A.Ncol + j] * A.unit;
            if (B == 0) write_result(A, t - 1, stt, stop_norm(A, L1), OT_VARIANT_TWOPASS);
            break;
        }
        // the queue of the next sweep is idle now (every block has left the previous column pass)
        if (B == 0 && tid == 0) A.queue[nxt] = 0;

        // ---- column pass over dynamically claimed 32-column chunks: lane <-> column, warps split rows
        const float* fh = A.fhi + nxt * A.M;
        const float* fr = A.frf + nxt * A.M;
        for (;;) {
            if (tid == 0) s_chunk = atomicAdd(&A.queue[cur], 1u);
            __syncthreads();
            const int chunk = (int)s_chunk;
            __syncthreads();
            if (chunk >= nchunks) break;
            const int c0 = chunk * 32;
            const int j = c0 + lane;
            const bool jv = j < A.Ncol;
            const float g = jv ? A.gc[cur * A.Ncol + j] : 0.f;
            const float2 yj = (OTF && jv) ? __ldg(A.Y + j) : make_float2(0.f, 0.f);
            float s = 0.f, sc = 0.f;   // compensated: n / OT_WARPS terms per thread
            if (jv) {
                for (int i = wid; i < A.M; i += OT_WARPS) {
                    float c;
                    if (OTF) {
                        const float2 xi = __ldg(A.X + i);
                        const float dx = xi.x - yj.x, dy = xi.y - yj.y;
                        c = fmaf(dx, dx, dy * dy);
                    } else {
                        c = __ldg(A.C + (long long)i * A.ld + j);
                    }
                    kahan_add(s, sc, ex2(fmaf(c, -A.kappa, fh[i]) + g) * fr[i]);
                }
            }
            s_col[wid][lane] = s - sc;
            __syncthreads();
            if (wid == 0) {
                int bad = 0;
                if (jv) {
                    double R2 = 0.0;
                    for (int w = 0; w < OT_WARPS; ++w) R2 += (double)s_col[w][lane];
                    R2 *= (double)A.cf[cur * A.Ncol + j];
                    if (R2 != R2) {
                        set_status(A.ctrl, OT_ERR_NONFINITE);
                    } else if (R2 > 1e-30 && R2 < 1e30) {
                        const double beta = (double)A.b[j] * inv_sb;
                        store_col(A, nxt, j, A.gam[cur * A.Ncol + j] - (double)lg2((float)(R2 / beta)));
                    } else {
                        bad = 1;
                    }
                }
                s_flag[lane] = bad;
            }
            __syncthreads();
            for (int l = 0; l < 32; ++l)
                if (s_flag[l]) column_fallback<OTF>(A, c0 + l, nxt, inv_sb, s_redf);
        }
        trace_mark(A, t, 3);
        if (!grid_sync(A.ctrl, G, A.timeout_ns, epoch)) { go = false; break; }
    }
    if (!args_ok) {
        if (B == 0) write_result(A, 0, OT_ERR_ARG, -1.0, OT_VARIANT_TWOPASS);
    } else if (!go) {
        fail_exit(A);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct WsLayout {
    size_t ctrl, phi, fhi, frf, gam, gc, cf, part, l1part, queue, acc, trace, total;
    int vstride;
    int pstride;
};

static WsLayout ws_layout(int M, int Ncol, int grid, bool fused) {
    WsLayout L;
    L.pstride = (Ncol + 3) & ~3;
    size_t o = 0;
    L.ctrl = o; o = align256_hd(o + sizeof(Ctrl));
    L.phi = o; o = align256_hd(o + sizeof(double) * 2 * (size_t)M);
    L.fhi = o; o = align256_hd(o + sizeof(float) * 2 * (size_t)M);
    L.frf = o; o = align256_hd(o + sizeof(float) * 2 * (size_t)M);
    L.gam = o; o = align256_hd(o + sizeof(double) * 2 * (size_t)Ncol);
    L.gc = o; o = align256_hd(o + sizeof(float) * 4 * (size_t)Ncol);   // also [2][Ncol] (hi, lo) pairs
    L.cf = o; o = align256_hd(o + sizeof(float) * 2 * (size_t)Ncol);
    L.part = o; o = align256_hd(o + (fused ? sizeof(float) * (size_t)grid * L.pstride : 0));
    L.l1part = o; o = align256_hd(o + sizeof(double) * (size_t)grid);
    L.queue = o; o = align256_hd(o + sizeof(unsigned) * 2);
    L.vstride = ((((Ncol + 2047) & ~2047) + 2) + 31) & ~31;   // whole 4 NT-column chunks + the L1 slot
    L.acc = o; o = align256_hd(o + (fused ? sizeof(double) * 3 * OT_ACC_COPIES * (size_t)L.vstride : 0));
    L.trace = o; o = align256_hd(o + sizeof(unsigned long long) * 8 * OT_TRACE_SWEEPS);
    L.total = o;
    return L;
}

static const int kFusedMaxCols = OT_BLOCK * 16;
static const int kFusedMaxRowsPerBlock = 128;
static const size_t kSmemBudget = 200 * 1024;

// Blocks of the persistent solvers: about four rows each, at most one per SM, and at most
// 128 up to 1024 rows, where the sweep is one band per block and the column exchange
// dominates (m = 1024 on this GPU: 6.48 us per sweep with 128 blocks, 6.91 with 152).
static int solver_grid(int M) {
    int sms = device_sms();
    if (sms <= 0) return 0;
    int g = (M + 3) / 4;
    if (g > sms) g = sms;
    if (M <= 1024 && g > 128) g = 128;
    if (g < 1) g = 1;
    return g;
}

static bool fused_ok(const SkArgs& A, int grid) {
    return A.C != nullptr && A.Ncol <= kFusedMaxCols && A.Ncol % 4 == 0 && A.ld == A.Ncol &&
           ((uintptr_t)A.C) % 16 == 0 && (A.M + grid - 1) / grid <= kFusedMaxRowsPerBlock &&
           (A.Ncol + grid - 1) / grid <= kFusedMaxRowsPerBlock;
}

size_t batch_single_ws_bytes(int m);

size_t solver_ws_bytes(int M, int Ncol, bool stored) {
    const bool fused = stored && Ncol <= kFusedMaxCols;   // partial buffer sized whenever it may be used
    const int grid = solver_grid(M);
    if (grid <= 0) return 0;
    size_t b = ws_layout(M, Ncol, grid, fused).total;
    if (stored && M == Ncol && Ncol > kFusedMaxCols && Ncol <= 8192) {   // the streaming route
        const size_t s = batch_single_ws_bytes(Ncol);
        b = s > b ? s : b;
    }
    return b;
}

template <typename K, typename... Args>
static int coop_launch_nt(K kernel, int grid, int nt, cudaStream_t st, size_t smem, Args... args) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return OT_ERR_CUDA;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, nt, smem) != cudaSuccess || nb < 1)
        return OT_ERR_UNSUPPORTED;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
    return e == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}

template <typename K, typename... Args>
static int coop_launch(K kernel, int grid, cudaStream_t st, size_t smem, Args... args) {
    return coop_launch_nt(kernel, grid, OT_BLOCK, st, smem, args...);
}

template <int CPT, int R>
static int launch_fused(SkArgs& A, int grid, cudaStream_t st) {
    const int rows_max = (A.M + grid - 1) / grid;
    const int nb_max = (rows_max + R - 1) / R;
    const size_t band_bytes = (size_t)R * A.Ncol * sizeof(float);
    A.rows_max = rows_max;
    A.cols_max = (A.Ncol + grid - 1) / grid;
    const size_t state = align256_hd(fused_rowstate_bytes(A.rows_max)) + fused_colstate_bytes(A.cols_max);
    A.resident = (nb_max <= OT_MAX_STAGES && nb_max * band_bytes + state <= kSmemBudget) ? 1 : 0;
    const int nstage = A.resident ? nb_max : 2;
    const size_t smem = (size_t)nstage * band_bytes + state;
    return coop_launch(sk_fused_kernel<CPT, R>, grid, st, smem, A, nstage);
}

template <int CPT, int R>
static int launch_bulk_r(SkArgs& A, int grid, cudaStream_t st) {
    A.rows_max = (A.M + grid - 1) / grid;
    const int nb_max = (A.rows_max + R - 1) / R;
    const size_t band_bytes = (size_t)R * A.Ncol * sizeof(float);
    const size_t state = align256_hd((size_t)(A.Ncol + 2) * sizeof(double)) +
                         align256_hd((size_t)3 * A.Ncol * sizeof(float)) + fused_rowstate_bytes(A.rows_max);
    A.resident = (nb_max <= OT_MAX_STAGES && nb_max * band_bytes + state <= kSmemBudget) ? 1 : 0;
    const int nstage = A.resident ? nb_max : 2;
    const size_t smem = (size_t)nstage * band_bytes + state;
    if (smem > 227 * 1024) return OT_ERR_UNSUPPORTED;
    return coop_launch(sk_bulk_kernel<CPT, R>, grid, st, smem, A, nstage);
}

// One grid barrier per sweep (bulk FP64 reduce-add of the column sums).
static int launch_bulk(SkArgs& A, int grid, cudaStream_t st) {
    const int cpt = (A.Ncol + OT_BLOCK - 1) / OT_BLOCK;
    const int rows_max = (A.M + grid - 1) / grid;
    if (cpt <= 4) return rows_max <= 8 ? launch_bulk_r<4, 8>(A, grid, st) : launch_bulk_r<4, 16>(A, grid, st);
    if (cpt <= 8) return launch_bulk_r<8, 8>(A, grid, st);
    return launch_bulk_r<16, 4>(A, grid, st);
}

// Ring kernel: NT threads, CPT columns per thread, bands of R rows, S ring stages.
template <int NT, int CPT, int R, int S>
static int launch_ring_t(SkArgs& A, int grid, cudaStream_t st) {
    A.rows_max = (A.M + grid - 1) / grid;
    const int nb_max = (A.rows_max + R - 1) / R;
    const size_t band_bytes = (size_t)R * A.Ncol * sizeof(float);
    const size_t state = align256_hd((size_t)(4 * NT + 2) * sizeof(double)) + (size_t)A.rows_max * 7 * sizeof(float);
    const size_t limit = 227 * 1024 - 4096;   // the opt-in maximum less the kernel's static shared memory
    const size_t res_bytes = align256_hd((size_t)nb_max * band_bytes);
    A.resident = (res_bytes + state <= limit) ? 1 : 0;
    const size_t smem = (A.resident ? res_bytes : align256_hd((size_t)S * band_bytes)) + state;
    if (smem > limit) return OT_ERR_UNSUPPORTED;
    return coop_launch_nt(sk_ring_kernel<NT, CPT, R, S>, grid, NT, st, smem, A);
}

static bool ring_ok(const SkArgs& A, int grid) {
    return A.C != nullptr && A.Ncol % 4 == 0 && A.ld == A.Ncol && ((uintptr_t)A.C) % 16 == 0 && A.Ncol <= 4096 &&
           !A.stop_l2 && (A.M + grid - 1) / grid <= 128;
}

template <int CPT, int R, int S>
static int launch_pp_t(SkArgs& A, int grid, cudaStream_t st) {
    A.rows_max = (A.M + grid - 1) / grid;
    if ((A.Ncol + grid - 1) / grid > 32) return OT_ERR_UNSUPPORTED;   // owned columns per block
    const int nb_max = (A.rows_max + R - 1) / R;
    const size_t band_bytes = (size_t)R * A.Ncol * sizeof(float);
    const size_t state = 2 * align256_hd((size_t)PP_G * CPT * sizeof(float)) +
                         align256_hd((size_t)A.rows_max * 7 * sizeof(float)) + 4 * 32 * sizeof(float);
    const size_t limit = 227 * 1024 - 8192;   // the opt-in maximum less the kernel's static shared memory
    const size_t res_bytes = align256_hd(2 * (size_t)((nb_max + 1) / 2) * band_bytes);
    A.resident = (res_bytes + state <= limit) ? 1 : 0;
    const size_t smem = (A.resident ? res_bytes : align256_hd(2 * (size_t)S * band_bytes)) + state;
    if (smem > limit) return OT_ERR_UNSUPPORTED;
    return coop_launch_nt(sk_pp_kernel<CPT, R, S>, grid, 2 * PP_G, st, smem, A);
}

// Up to 1024 columns the single-group ring kernel (one barrier per sweep, bulk FP64 adds at L2)
// is faster: the column exchange dominates small sweeps.  Wider costs take the ping-pong kernel.
static int launch_ring(SkArgs& A, int grid, cudaStream_t st) {
    if (A.Ncol <= 1024) return launch_ring_t<256, 4, 8, 3>(A, grid, st);
    if (A.Ncol <= 2048) return launch_pp_t<8, 4, 3>(A, grid, st);
    return launch_pp_t<16, 2, 2>(A, grid, st);
}

size_t batch_single_ws_bytes(int m);
int batch_single_solve(int m, int N, const float* G, int ld, const float* a, const float* b, const ot_options* opt,
                       double* w, double* z, ot_result* out, void* workspace, size_t ws_bytes, cudaStream_t st);

// A square stored cost too wide for the resident kernels (4096 < columns <= 8192,
// rows 16-byte aligned) streams through the batch kernel: bulk-copy pipeline,
// one read of the cost per sweep, compensated column sums.
static bool streaming_ok(const SkArgs& A, int grid, const ot_options* o) {
    return A.C != nullptr && !fused_ok(A, grid) && A.M == A.Ncol && A.Ncol > kFusedMaxCols && A.Ncol <= 8192 &&
           A.ld % 4 == 0 && ((uintptr_t)A.C) % 16 == 0 && o->stop_norm == OT_STOP_L1_FULL && o->debug_flags == 0;
}

int run_solver(SkArgs A, void* ws, size_t ws_bytes, cudaStream_t st) {
    const bool stored = A.C != nullptr;
    const int grid = solver_grid(A.M);
    if (grid <= 0) return OT_ERR_CUDA;
    const bool fused = fused_ok(A, grid);
    const WsLayout L = ws_layout(A.M, A.Ncol, grid, stored && A.Ncol <= kFusedMaxCols);
    if (ws == nullptr || ws_bytes < L.total) return OT_ERR_WORKSPACE;
    if (((uintptr_t)ws) % 256 != 0) return OT_ERR_WORKSPACE;
    char* w = (char*)ws;
    A.ctrl = (Ctrl*)(w + L.ctrl);
    A.phi = (double*)(w + L.phi);
    A.fhi = (float*)(w + L.fhi);
    A.frf = (float*)(w + L.frf);
    A.gam = (double*)(w + L.gam);
    A.gc = (float*)(w + L.gc);
    A.cf = (float*)(w + L.cf);
    A.part = (float*)(w + L.part);
    A.l1part = (double*)(w + L.l1part);
    A.queue = (unsigned*)(w + L.queue);
    A.acc = (double*)(w + L.acc);
    A.vstride = L.vstride;
    A.trace = (A.debug_flags & OT_DEBUG_TRACE) ? (unsigned long long*)(w + L.trace) : nullptr;
    A.pstride = L.pstride;
    if (cudaMemsetAsync(A.ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return OT_ERR_CUDA;
    if (fused && cudaMemsetAsync(A.acc, 0, sizeof(double) * 3 * OT_ACC_COPIES * (size_t)L.vstride, st) != cudaSuccess)
        return OT_ERR_CUDA;
    if (!fused) {
        A.rows_max = (A.M + grid - 1) / grid;
        const size_t smem = fused_rowstate_bytes(A.rows_max);
        if (smem > kSmemBudget) return OT_ERR_UNSUPPORTED;
        return stored ? coop_launch(sk_twopass_kernel<false>, grid, st, smem, A)
                      : coop_launch(sk_twopass_kernel<true>, grid, st, smem, A);
    }
    if (ring_ok(A, grid) && !(A.debug_flags & (OT_DEBUG_NO_CLUSTER | OT_DEBUG_NO_RING))) {
        const int rc = launch_ring(A, grid, st);
        if (rc != OT_ERR_UNSUPPORTED) return rc;
    }
    const int cpt = (A.Ncol + OT_BLOCK - 1) / OT_BLOCK;
    // the cluster kernel updates every column in every block: worth it while Ncol <= 2048
    // one barrier per sweep pays while the per-sweep column-sum vector is small
    if (!(A.debug_flags & OT_DEBUG_NO_CLUSTER) && A.Ncol <= 2048) {
        const int rc = launch_bulk(A, grid, st);
        if (rc != OT_ERR_UNSUPPORTED) return rc;
    }
    const int rows_max = (A.M + grid - 1) / grid;
    if (cpt <= 4) return rows_max <= 8 ? launch_fused<4, 8>(A, grid, st) : launch_fused<4, 16>(A, grid, st);
    if (cpt <= 8) return launch_fused<8, 8>(A, grid, st);
    return launch_fused<16, 4>(A, grid, st);
}

static bool opt_ok(const ot_options* o) {
    return o && o->eps > 0.f && o->max_iter >= 1 && o->check_every >= 1 && o->tol_l1 >= 0.0 &&
           (o->stop_norm == OT_STOP_L1_FULL || o->stop_norm == OT_STOP_L2_ROW) &&
           o->precision == OT_FP32_LOG && o->tile_override == 0;
}

static SkArgs base_args(const ot_options* o) {
    SkArgs A;
    memset(&A, 0, sizeof(A));
    const double e = (double)o->eps;
    A.kappa = (float)(1.0 / (e * OT_LN2));
    A.unit = e * OT_LN2;
    A.tol = o->tol_l1;
    A.max_iter = o->max_iter;
    A.check_every = o->check_every;
    A.timeout_ns = o->timeout_ns ? o->timeout_ns : 10000000000ull;
    A.warm = o->warm_start ? 1 : 0;
    A.debug_flags = o->debug_flags;
    A.stop_l2 = o->stop_norm == OT_STOP_L2_ROW ? 1 : 0;
    A.l2_scale = 1.0;
    return A;
}

}  // namespace cyc

using namespace cyc;

extern "C" int ot_sinkhorn_reduced(int m, int N, const float* a_base, const float* b_base, const float* G,
                                   const ot_options* opt, double* w, double* z, ot_result* out, void* workspace,
                                   size_t ws_bytes, void* stream) {
    if (m <= 0 || N <= 0 || !a_base || !b_base || !G || !w || !z || !out || !opt_ok(opt)) return OT_ERR_ARG;
    if (((uintptr_t)G) % 16 != 0) return OT_ERR_ARG;
    SkArgs A = base_args(opt);
    A.M = m;
    A.Ncol = m;
    A.ld = m;
    A.C = G;
    A.a = a_base;
    A.b = b_base;
    // the solver runs with unit-mass marginals; the paper's w (mass 1/N) is f - eps log N
    A.f_shift = -(double)opt->eps * log((double)N);
    A.l2_scale = 1.0 / (double)N;   // L2 rule: the row error of the mass-1/N reduced problem
    A.f_out = w;
    A.g_out = z;
    A.res = out;
    const int grid = solver_grid(A.M);
    if (grid > 0 && streaming_ok(A, grid, opt))
        return batch_single_solve(m, N, G, m, a_base, b_base, opt, w, z, out, workspace, ws_bytes,
                                  (cudaStream_t)stream);
    return run_solver(A, workspace, ws_bytes, (cudaStream_t)stream);
}

extern "C" int ot_sinkhorn_full(int n, const float* a, const float* b, const float* C, const float* X,
                                const float* Y, const ot_options* opt, double* f, double* g, ot_result* out,
                                void* workspace, size_t ws_bytes, void* stream) {
    if (n <= 0 || !a || !b || !f || !g || !out || !opt_ok(opt)) return OT_ERR_ARG;
    if (!C && (!X || !Y)) return OT_ERR_ARG;
    if (C && ((uintptr_t)C) % 16 != 0) return OT_ERR_ARG;
    SkArgs A = base_args(opt);
    A.M = n;
    A.Ncol = n;
    A.ld = n;
    A.C = C;
    A.X = (const float2*)X;
    A.Y = (const float2*)Y;
    A.a = a;
    A.b = b;
    A.f_shift = 0.0;
    A.f_out = f;
    A.g_out = g;
    A.res = out;
    const int grid = solver_grid(A.M);
    if (grid > 0 && streaming_ok(A, grid, opt))
        return batch_single_solve(n, 1, C, n, a, b, opt, f, g, out, workspace, ws_bytes, (cudaStream_t)stream);
    return run_solver(A, workspace, ws_bytes, (cudaStream_t)stream);
}
