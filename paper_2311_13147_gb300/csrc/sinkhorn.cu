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
// running max).  Rows whose sum leaves [1e-30, 1e30] (first sweep, far warm
// starts) are redone with an explicit max shift.
//
// Fused single-read sweep (narrow problems, Ncol <= 4096): a block owns a
// contiguous row range and keeps a band of R rows x all columns in registers.
// After the band's row sums give phi_new, the column contributions of the same
// entries are u_i * e_ij with u_i = alpha_i / S_i -- the row pass's
// exponentials reused, because 2^(phi_new_i + gamma_j - c_ij) = e_ij * alpha_i / S_i.
// One cost read and ONE exp2 per entry per sweep.  Per-block column partials
// go to the workspace; after a grid barrier the column owners reduce them in
// a fixed order (FP64) and update gamma.  Second barrier, next sweep.
//
// Two-pass sweep (wide or on-the-fly costs): row pass then column pass, each
// a full sweep over the cost (two exp2 per entry), no partials.
//
// Potentials are carried in FP64 (2 values per row/column per sweep) and
// split into FP32 hi + a FP32 factor 2^lo for the inner loops, which are pure
// FP32: an FP32 potential alone would bias every plan row by up to
// ulp(phi)/2 relative, above a 1e-6 marginal target when |f|/eps ~ 100.
#include <math.h>

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
    unsigned long long* trace;    // [kTraceSweeps][8] phase timestamps, or null
    int pstride;
};

// Buffers: the state after s iterations lives in phi[s & 1] and gam[s & 1].
// Sweep t reads state t-1 and writes state t.

#define OT_TRACE_SWEEPS 256
__device__ __forceinline__ void trace_mark(const SkArgs& A, int t, int slot) {
    if (A.trace != nullptr && blockIdx.x == 0 && threadIdx.x == 0 && t < OT_TRACE_SWEEPS)
        A.trace[t * 8 + slot] = globaltimer();
}

__device__ __forceinline__ bool sum_ok(float s) { return s > 1e-30f && s < 1e30f; }

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
    float hi = (float)g;
    A.gam[buf * A.Ncol + j] = g;
    A.gc[buf * A.Ncol + j] = hi;
    A.cf[buf * A.Ncol + j] = ex2((float)(g - (double)hi));
}

__device__ __forceinline__ void store_row(const SkArgs& A, int buf, int i, double p) {
    float hi = (float)p;
    A.phi[buf * A.M + i] = p;
    A.fhi[buf * A.M + i] = hi;
    A.frf[buf * A.M + i] = ex2((float)(p - (double)hi));
}

// Write the returned state (rows and columns from buffer `buf`).
__device__ void write_outputs(const SkArgs& A, int buf, int r_beg, int r_end, int c_beg, int c_end) {
    for (int i = r_beg + threadIdx.x; i < r_end; i += OT_BLOCK)
        A.f_out[i] = A.phi[buf * A.M + i] * A.unit + A.f_shift;
    for (int j = c_beg + threadIdx.x; j < c_end; j += OT_BLOCK) A.g_out[j] = A.gam[buf * A.Ncol + j] * A.unit;
}

// Sum of the per-block L1 partials, all threads loading in parallel, fixed order.
__device__ double total_l1(const SkArgs& A, double* s_dred) {
    double v = 0.0;
    for (int b2 = threadIdx.x; b2 < gridDim.x; b2 += OT_BLOCK) v += ((volatile double*)A.l1part)[b2];
    return block_sum_d(v, s_dred);
}

// Stopping rule on the state after `done` iterations; returns the status or -1 to continue.
__device__ __forceinline__ int stop_status(const SkArgs& A, int done, double L1) {
    if (done < 1) return -1;
    if (L1 != L1) return OT_ERR_NONFINITE;
    if (done % A.check_every == 0 && L1 <= A.tol) return OT_OK;
    if (done >= A.max_iter) return OT_ERR_NOT_CONVERGED;
    return -1;
}

__device__ void write_result(const SkArgs& A, int iters, int status, double l1) {
    if (threadIdx.x == 0) {
        A.res->iters = iters;
        A.res->status = status;
        A.res->marg_l1 = l1;
        A.res->marg_l2_col = -1.0;
        A.res->value = 0.0;
        A.res->transport_cost = 0.0;
        A.res->marg_l1_col = -1.0;
    }
}

__device__ void fail_exit(const SkArgs& A) {
    if (threadIdx.x == 0) {
        A.res->iters = -1;
        A.res->status = ld_volatile_int(&A.ctrl->status);
    }
}

// Column update from a finished column sum R (true sum, column factor included):
// gamma_new = gamma_old - log2(R / beta_j), read from buffer ob, written to nb.
// Returns false if R is outside the safe range (caller falls back).
__device__ __forceinline__ bool column_update(const SkArgs& A, int ob, int nb, int j, double R, double inv_sb) {
    if (R != R) {
        set_status(A.ctrl, OT_ERR_NONFINITE);
        return true;
    }
    if (!(R > 1e-30 && R < 1e30)) return false;
    const double beta = (double)A.b[j] * inv_sb;
    const float d = lg2((float)(R / beta));
    store_col(A, nb, j, A.gam[ob * A.Ncol + j] - (double)d);
    return true;
}

// Robust column update with an explicit max shift over the whole column,
// from the new row potentials (buffer nb).  Whole block, one column.
template <bool OTF>
__device__ void column_fallback(const SkArgs& A, int j, int nb, double inv_sb, float* s_redf) {
    // row potentials and the new column potential both live in buffer nb
    float mx = -INFINITY;
    const float* fh = A.fhi + nb * A.M;
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
        s += ex2(fmaf(c, -A.kappa, fh[i]) - m2) * A.frf[nb * A.M + i];
    }
    s = warp_sum(s);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_redf[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int w = 0; w < OT_WARPS; ++w) tot += s_redf[w];
        const double beta = (double)A.b[j] * inv_sb;
        if (!(tot > 0.f) || !(m2 > -INFINITY)) {
            set_status(A.ctrl, OT_ERR_NONFINITE);
        } else {
            // gamma_new = log2 beta - (m2 + log2 tot)
            store_col(A, nb, j, (double)lg2((float)beta) - (double)m2 - (double)lg2(tot));
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Fused single-read kernel (Ncol <= OT_BLOCK * CPT)
// ---------------------------------------------------------------------------

// Per-row values the band epilogue needs, loaded at the start of the band so
// their latency hides behind the band's exponentials.
struct RowPre {
    float alpha, fhi, frf;
    double phi;
};

template <int CPT, int R, bool SAFE>
__device__ __forceinline__ void fused_band(const SkArgs& A, int rb, int nr, int cur, int nxt, double inv_sa,
                                           const float (&gcr)[CPT], const float (&cfr)[CPT], float (&e)[R][CPT],
                                           double& l1, float (*s_red)[R], float* s_F, float* s_u, int* s_bad) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    RowPre pre = {1.f, 0.f, 1.f, 0.0};
    if (tid < nr) {
        const int row = rb + tid;
        pre.alpha = (float)((double)A.a[row] * inv_sa);
        if (!SAFE) {
            pre.fhi = A.fhi[cur * A.M + row];
            pre.frf = A.frf[cur * A.M + row];
            pre.phi = A.phi[cur * A.M + row];
        }
    }
    // 1. exponents x = gamma_j - c_ij (+ phi_i when not SAFE); invalid rows skipped (uniform branch)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r < nr) {
            const float* crow = A.C + (long long)(rb + r) * A.ld;
            const float F = SAFE ? 0.f : A.fhi[cur * A.M + rb + r];
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const int j = tid + q * OT_BLOCK;
                e[r][q] = (j < A.Ncol) ? fmaf(__ldg(crow + j), -A.kappa, gcr[q]) + F : -INFINITY;
            }
        }
    }
    if (SAFE) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r < nr) {
                float mx = e[r][0];
#pragma unroll
                for (int q = 1; q < CPT; ++q) mx = fmaxf(mx, e[r][q]);
                mx = warp_max(mx);
                if (lane == 0) s_red[wid][r] = mx;
            }
        }
        __syncthreads();
        if (tid < nr) {
            float mx = s_red[0][tid];
            for (int w = 1; w < OT_WARPS; ++w) mx = fmaxf(mx, s_red[w][tid]);
            s_F[tid] = (mx > -INFINITY) ? -mx : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r < nr) {
                const float F = s_F[r];
#pragma unroll
                for (int q = 0; q < CPT; ++q) e[r][q] += F;
            }
        }
    }
    // 2. e = 2^x * colfactor, row partial sums
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r < nr) {
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                e[r][q] = ex2(e[r][q]) * cfr[q];
                s += e[r][q];
            }
            s = warp_sum(s);
            if (lane == 0) s_red[wid][r] = s;
        } else {
#pragma unroll
            for (int q = 0; q < CPT; ++q) e[r][q] = 0.f;
        }
    }
    __syncthreads();
    // 3. row epilogue: one thread per row
    if (tid < R) {
        float u = 0.f;
        if (tid < nr) {
            const int row = rb + tid;
            float S = 0.f;
#pragma unroll
            for (int w = 0; w < OT_WARPS; ++w) S += s_red[w][tid];
            const float alpha = pre.alpha;
            double pnew;
            if (!SAFE) {
                // L1 term of the current state: |S * 2^lo - alpha|
                l1 += fabs((double)fmaf(S, pre.frf - 1.0f, S - alpha));
                pnew = (double)pre.fhi - (double)lg2(S / alpha);
            } else {
                pnew = (double)s_F[tid] - (double)lg2(S / alpha);
            }
            if (sum_ok(S)) {
                store_row(A, nxt, row, pnew);
                u = alpha / S;
            } else {
                *s_bad = 1;
            }
        }
        s_u[tid] = u;
    }
    __syncthreads();
}

template <int CPT, int R>
__global__ void __launch_bounds__(OT_BLOCK, 1) sk_fused_kernel(SkArgs A) {
    __shared__ float s_red[OT_WARPS][R];
    __shared__ float s_F[R];
    __shared__ float s_u[R];
    __shared__ int s_bad;
    __shared__ double s_dred[OT_WARPS];
    __shared__ float s_redf[OT_WARPS];
    __shared__ int s_flag_cols[64];
    __shared__ int s_nflag;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int B = blockIdx.x, G = gridDim.x;
    const int r_beg = (int)((long long)A.M * B / G), r_end = (int)((long long)A.M * (B + 1) / G);
    const int c_beg = (int)((long long)A.Ncol * B / G), c_end = (int)((long long)A.Ncol * (B + 1) / G);

    double inv_sa, inv_sb;
    if (!prologue_sums(A, inv_sa, inv_sb, s_dred)) {
        if (B == 0) write_result(A, 0, OT_ERR_ARG, -1.0);
        return;
    }
    for (int j = c_beg + tid; j < c_end; j += OT_BLOCK) store_col(A, 0, j, A.warm ? A.g_out[j] / A.unit : 0.0);
    if (tid == 0) { s_bad = 0; s_nflag = 0; }
    if ((A.debug_flags & OT_DEBUG_WITHHOLD_ARRIVAL) && B == 0) {
        withhold_arrival(A.ctrl, A.timeout_ns);
        fail_exit(A);
        return;
    }
    if (!grid_sync(A.ctrl, G, A.timeout_ns)) { fail_exit(A); return; }

    for (int t = 1;; ++t) {
        const int cur = (t - 1) & 1, nxt = cur ^ 1;
        trace_mark(A, t, 0);
        float gcr[CPT], cfr[CPT], acc[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int j = tid + q * OT_BLOCK;
            const bool v = j < A.Ncol;
            gcr[q] = v ? A.gc[cur * A.Ncol + j] : 0.f;
            cfr[q] = v ? A.cf[cur * A.Ncol + j] : 0.f;
            acc[q] = 0.f;
        }
        double l1 = 0.0;
        float e[R][CPT];
        for (int rb = r_beg; rb < r_end; rb += R) {
            const int nr = min(R, r_end - rb);
            if (t == 1) {
                fused_band<CPT, R, true>(A, rb, nr, cur, nxt, inv_sa, gcr, cfr, e, l1, s_red, s_F, s_u, &s_bad);
            } else {
                fused_band<CPT, R, false>(A, rb, nr, cur, nxt, inv_sa, gcr, cfr, e, l1, s_red, s_F, s_u, &s_bad);
            }
            if (s_bad) {   // uniform: read after the band's final __syncthreads
                __syncthreads();
                if (tid == 0) s_bad = 0;
                double dummy = 0.0;
                fused_band<CPT, R, true>(A, rb, nr, cur, nxt, inv_sa, gcr, cfr, e, dummy, s_red, s_F, s_u, &s_bad);
                if (s_bad) {
                    // still out of range after the max shift: non-finite input
                    if (tid == 0) { set_status(A.ctrl, OT_ERR_NONFINITE); s_bad = 0; }
                    __syncthreads();
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < nr) {
                    const float u = s_u[r];
#pragma unroll
                    for (int q = 0; q < CPT; ++q) acc[q] = fmaf(u, e[r][q], acc[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int j = tid + q * OT_BLOCK;
            if (j < A.Ncol) A.part[(long long)B * A.pstride + j] = acc[q];
        }
        l1 = block_sum_d(l1, s_dred);
        if (tid == 0) A.l1part[B] = l1;
        trace_mark(A, t, 1);
        if (!grid_sync(A.ctrl, G, A.timeout_ns)) { fail_exit(A); return; }
        trace_mark(A, t, 2);

        // ---- column phase for owned columns (one warp per column), writes buffer nxt
        for (int j = c_beg + wid; j < c_end; j += OT_WARPS) {
            double s = 0.0;
            for (int b2 = lane; b2 < G; b2 += 32) s += (double)A.part[(long long)b2 * A.pstride + j];
            s = warp_sum(s);
            if (lane == 0) {
                if (!column_update(A, cur, nxt, j, s, inv_sb)) {
                    const int k = atomicAdd(&s_nflag, 1);
                    if (k < 64) s_flag_cols[k] = j;
                    else set_status(A.ctrl, OT_ERR_NONFINITE);
                }
            }
        }
        // ---- stopping rule on the state after iteration t-1 (overlaps the column phase)
        const double L1 = total_l1(A, s_dred);
        const int st = stop_status(A, t - 1, L1);
        if (st >= 0) {
            write_outputs(A, cur, r_beg, r_end, c_beg, c_end);
            if (B == 0) write_result(A, t - 1, st, L1);
            return;
        }
        const int nflag = min(s_nflag, 64);
        __syncthreads();
        if (tid == 0) s_nflag = 0;
        for (int k = 0; k < nflag; ++k) column_fallback<false>(A, s_flag_cols[k], nxt, inv_sb, s_redf);
        trace_mark(A, t, 3);
        if (!grid_sync(A.ctrl, G, A.timeout_ns)) { fail_exit(A); return; }
    }
}

// ---------------------------------------------------------------------------
// Two-pass kernel (any width; stored or on-the-fly cost)
// ---------------------------------------------------------------------------

#define WR 8   // rows per band in the two-pass row phase

// Row phase for a band of up to WR rows: S_r = sum_j 2^(F_r + gamma_j - c_rj) * cf_j.
// SAFE: F_r = -max_j(gamma_j - c_rj) (extra pass).  Writes phi_new; adds L1.
template <bool OTF, bool SAFE>
__device__ void twopass_row_band(const SkArgs& A, int rb, int nr, int cur, int nxt, double inv_sa, double& l1,
                                 float (*s_red)[WR], float* s_F, int* s_bad) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const float* gcp = A.gc + cur * A.Ncol;
    const float* cfp = A.cf + cur * A.Ncol;
    RowPre pre = {1.f, 0.f, 1.f, 0.0};
    if (tid < nr) {
        const int row = rb + tid;
        pre.alpha = (float)((double)A.a[row] * inv_sa);
        if (!SAFE) {
            pre.fhi = A.fhi[cur * A.M + row];
            pre.frf = A.frf[cur * A.M + row];
        }
    }
    float F[WR];
    float2 xr[WR];
    const float* crow[WR];
#pragma unroll
    for (int r = 0; r < WR; ++r) {
        const int row = rb + (r < nr ? r : 0);
        xr[r] = OTF ? __ldg(A.X + row) : make_float2(0.f, 0.f);
        crow[r] = OTF ? nullptr : A.C + (long long)row * A.ld;
        F[r] = (!SAFE && r < nr) ? A.fhi[cur * A.M + row] : 0.f;
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
    float s[WR];
#pragma unroll
    for (int r = 0; r < WR; ++r) s[r] = 0.f;
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
                s[r] += ex2(fmaf(c, -A.kappa, g) + F[r]) * cfj;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < WR; ++r) {
        const float v = warp_sum(s[r]);
        if (lane == 0) s_red[wid][r] = v;
    }
    __syncthreads();
    if (tid < nr) {
        const int row = rb + tid;
        float S = 0.f;
        for (int w = 0; w < OT_WARPS; ++w) S += s_red[w][tid];
        const float alpha = pre.alpha;
        double pnew;
        if (!SAFE) {
            l1 += fabs((double)fmaf(S, pre.frf - 1.0f, S - alpha));
            pnew = (double)pre.fhi - (double)lg2(S / alpha);
        } else {
            pnew = (double)s_F[tid] - (double)lg2(S / alpha);
        }
        if (sum_ok(S)) store_row(A, nxt, row, pnew);
        else *s_bad = 1;
    }
    __syncthreads();
}

template <bool OTF>
__global__ void __launch_bounds__(OT_BLOCK, 1) sk_twopass_kernel(SkArgs A) {
    __shared__ float s_red[OT_WARPS][WR];
    __shared__ float s_F[WR];
    __shared__ int s_bad;
    __shared__ double s_dred[OT_WARPS];
    __shared__ float s_redf[OT_WARPS];
    __shared__ float s_col[OT_WARPS][32];
    __shared__ int s_flag[32];

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int B = blockIdx.x, G = gridDim.x;
    const int r_beg = (int)((long long)A.M * B / G), r_end = (int)((long long)A.M * (B + 1) / G);
    // columns are handed out in chunks of 32 (one lane per column)
    const int nchunks = (A.Ncol + 31) / 32;
    const int k_beg = (int)((long long)nchunks * B / G), k_end = (int)((long long)nchunks * (B + 1) / G);
    const int c_beg = min(A.Ncol, k_beg * 32), c_end = min(A.Ncol, k_end * 32);

    double inv_sa, inv_sb;
    if (!prologue_sums(A, inv_sa, inv_sb, s_dred)) {
        if (B == 0) write_result(A, 0, OT_ERR_ARG, -1.0);
        return;
    }
    for (int j = c_beg + tid; j < c_end; j += OT_BLOCK) store_col(A, 0, j, A.warm ? A.g_out[j] / A.unit : 0.0);
    if (tid == 0) s_bad = 0;
    if ((A.debug_flags & OT_DEBUG_WITHHOLD_ARRIVAL) && B == 0) {
        withhold_arrival(A.ctrl, A.timeout_ns);
        fail_exit(A);
        return;
    }
    if (!grid_sync(A.ctrl, G, A.timeout_ns)) { fail_exit(A); return; }

    for (int t = 1;; ++t) {
        const int cur = (t - 1) & 1, nxt = cur ^ 1;
        trace_mark(A, t, 0);
        double l1 = 0.0;
        for (int rb = r_beg; rb < r_end; rb += WR) {
            const int nr = min(WR, r_end - rb);
            if (t == 1) twopass_row_band<OTF, true>(A, rb, nr, cur, nxt, inv_sa, l1, s_red, s_F, &s_bad);
            else twopass_row_band<OTF, false>(A, rb, nr, cur, nxt, inv_sa, l1, s_red, s_F, &s_bad);
            if (s_bad) {
                __syncthreads();
                if (tid == 0) s_bad = 0;
                double dummy = 0.0;
                twopass_row_band<OTF, true>(A, rb, nr, cur, nxt, inv_sa, dummy, s_red, s_F, &s_bad);
                if (s_bad) {
                    if (tid == 0) { set_status(A.ctrl, OT_ERR_NONFINITE); s_bad = 0; }
                    __syncthreads();
                }
            }
        }
        l1 = block_sum_d(l1, s_dred);
        if (tid == 0) A.l1part[B] = l1;
        trace_mark(A, t, 1);
        if (!grid_sync(A.ctrl, G, A.timeout_ns)) { fail_exit(A); return; }
        trace_mark(A, t, 2);

        const double L1 = total_l1(A, s_dred);
        const int st = stop_status(A, t - 1, L1);
        if (st >= 0) {
            write_outputs(A, cur, r_beg, r_end, c_beg, c_end);
            if (B == 0) write_result(A, t - 1, st, L1);
            return;
        }

        // ---- column pass: lane <-> column, warps split the rows; writes buffer nxt
        const float* fh = A.fhi + nxt * A.M;
        const float* fr = A.frf + nxt * A.M;
        for (int c0 = c_beg; c0 < c_end; c0 += 32) {
            const int j = c0 + lane;
            const bool jv = j < c_end;
            const float g = jv ? A.gc[cur * A.Ncol + j] : 0.f;
            const float2 yj = (OTF && jv) ? __ldg(A.Y + j) : make_float2(0.f, 0.f);
            float s = 0.f;
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
                    s += ex2(fmaf(c, -A.kappa, fh[i]) + g) * fr[i];
                }
            }
            s_col[wid][lane] = s;
            __syncthreads();
            if (wid == 0) {
                int bad = 0;
                if (jv) {
                    double R = 0.0;
                    for (int w = 0; w < OT_WARPS; ++w) R += (double)s_col[w][lane];
                    R *= (double)A.cf[cur * A.Ncol + j];
                    bad = !column_update(A, cur, nxt, j, R, inv_sb);
                }
                s_flag[lane] = bad;
            }
            __syncthreads();
            for (int l = 0; l < 32; ++l)
                if (s_flag[l]) column_fallback<OTF>(A, c0 + l, nxt, inv_sb, s_redf);
        }
        trace_mark(A, t, 3);
        if (!grid_sync(A.ctrl, G, A.timeout_ns)) { fail_exit(A); return; }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WsLayout {
    size_t ctrl, phi, fhi, frf, gam, gc, cf, part, l1part, trace, total;
    int pstride;
};

static WsLayout ws_layout(int M, int Ncol, int grid, bool fused) {
    WsLayout L;
    L.pstride = (Ncol + 3) & ~3;
    size_t o = 0;
    L.ctrl = o; o = align256(o + sizeof(Ctrl));
    L.phi = o; o = align256(o + sizeof(double) * 2 * (size_t)M);
    L.fhi = o; o = align256(o + sizeof(float) * 2 * (size_t)M);
    L.frf = o; o = align256(o + sizeof(float) * 2 * (size_t)M);
    L.gam = o; o = align256(o + sizeof(double) * 2 * (size_t)Ncol);
    L.gc = o; o = align256(o + sizeof(float) * 2 * (size_t)Ncol);
    L.cf = o; o = align256(o + sizeof(float) * 2 * (size_t)Ncol);
    L.part = o; o = align256(o + (fused ? sizeof(float) * (size_t)grid * L.pstride : 0));
    L.l1part = o; o = align256(o + sizeof(double) * (size_t)grid);
    L.trace = o; o = align256(o + sizeof(unsigned long long) * 8 * OT_TRACE_SWEEPS);
    L.total = o;
    return L;
}

static const int kFusedMaxCols = OT_BLOCK * 16;

static int solver_grid(int M) {
    int sms = device_sms();
    if (sms <= 0) return 0;
    int g = (M + 3) / 4;
    if (g > sms) g = sms;
    if (g < 1) g = 1;
    return g;
}

size_t solver_ws_bytes(int M, int Ncol, bool stored) {
    const bool fused = stored && Ncol <= kFusedMaxCols;
    const int grid = solver_grid(M);
    if (grid <= 0) return 0;
    return ws_layout(M, Ncol, grid, fused).total;
}

template <typename K>
static int coop_launch(K kernel, int grid, SkArgs& A, cudaStream_t st) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, OT_BLOCK, 0) != cudaSuccess || nb < 1)
        return OT_ERR_UNSUPPORTED;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(OT_BLOCK);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, A);
    return e == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}

int run_solver(SkArgs A, void* ws, size_t ws_bytes, cudaStream_t st) {
    const bool stored = A.C != nullptr;
    const bool fused = stored && A.Ncol <= kFusedMaxCols;
    const int grid = solver_grid(A.M);
    if (grid <= 0) return OT_ERR_CUDA;
    const WsLayout L = ws_layout(A.M, A.Ncol, grid, fused);
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
    A.trace = (A.debug_flags & OT_DEBUG_TRACE) ? (unsigned long long*)(w + L.trace) : nullptr;
    A.pstride = L.pstride;
    if (cudaMemsetAsync(A.ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return OT_ERR_CUDA;
    if (!fused) {
        return stored ? coop_launch(sk_twopass_kernel<false>, grid, A, st)
                      : coop_launch(sk_twopass_kernel<true>, grid, A, st);
    }
    const int cpt = (A.Ncol + OT_BLOCK - 1) / OT_BLOCK;
    if (cpt <= 1) return coop_launch(sk_fused_kernel<1, 16>, grid, A, st);
    if (cpt <= 2) return coop_launch(sk_fused_kernel<2, 16>, grid, A, st);
    if (cpt <= 4) return coop_launch(sk_fused_kernel<4, 16>, grid, A, st);
    if (cpt <= 8) return coop_launch(sk_fused_kernel<8, 8>, grid, A, st);
    return coop_launch(sk_fused_kernel<16, 4>, grid, A, st);
}

static bool opt_ok(const ot_options* o) {
    return o && o->eps > 0.f && o->max_iter >= 1 && o->check_every >= 1 && o->tol_l1 >= 0.0 &&
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
    A.f_out = w;
    A.g_out = z;
    A.res = out;
    return run_solver(A, workspace, ws_bytes, (cudaStream_t)stream);
}

extern "C" int ot_sinkhorn_full(int n, const float* a, const float* b, const float* C, const float* X,
                                const float* Y, const ot_options* opt, double* f, double* g, ot_result* out,
                                void* workspace, size_t ws_bytes, void* stream) {
    if (n <= 0 || !a || !b || !f || !g || !out || !opt_ok(opt)) return OT_ERR_ARG;
    if (!C && (!X || !Y)) return OT_ERR_ARG;
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
    return run_solver(A, workspace, ws_bytes, (cudaStream_t)stream);
}
