// Batches of independent cyclic problems (uneven m and N): fold and cyclic
// Sinkhorn for all of them in one persistent launch each.
//
// Solver (Algorithm 2 per problem, log domain, the same iteration and stopping
// rule as ot_sinkhorn_reduced).  Two bounded grid barriers per sweep:
//
//  row phase    The rows of the still-active problems form one index space
//               weighted by row length; every block takes a contiguous,
//               equally weighted range of it (recomputed identically in every
//               block each sweep, so finished problems free their share).  A
//               band of R rows is streamed twice from global memory (float4,
//               coalesced; the second read hits L1/L2): pass 1 forms the row
//               sums and the new row potentials, pass 2 the column
//               contributions u_i * e_ij, accumulated in shared memory per
//               problem segment and added into the problem's column sums with
//               FP32 reductions (a problem is split over few blocks, so each
//               sum receives few terms).  The row L1 terms go to a per-problem
//               FP64 accumulator.
//  column phase The columns of the active problems are split the same way;
//               each column's potential is updated from its sum (FP64), the
//               sum is cleared, and the block holding a problem's column 0
//               applies the stopping rule: a finished problem's state (after
//               t-1 iterations) is frozen and recorded.
//
// When no problem is active, every block writes the outputs of its share.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace cyc {

int device_sms();

#define OT_BATCH_MAX 1024     // problems per batch
#define OT_BATCH_MAXM 8192    // largest block size
#define OT_BT 512             // threads per block
#define OT_BW (OT_BT / 32)
#define OT_BR 4               // rows per band

struct BatchArgs {
    int count;
    long long total_m;
    const float* G;
    const float* a;
    const float* b;
    double tol;
    int max_iter;
    unsigned long long timeout_ns;
    int warm;
    double* w_out;
    double* z_out;
    ot_result* res;
    // workspace
    Ctrl* ctrl;
    const ot_problem_desc* desc;   // [count]
    double* inv_sa;                // [count]
    double* inv_sb;                // [count]
    int* active;                   // [count]
    int* iters;                    // [count]
    double* l1acc;                 // [2][count]
    double* phi;                   // [2][total_m]
    float* fhi;                    // [2][total_m]
    float* frf;                    // [2][total_m]
    double* gam;                   // [total_m]
    float* gc;                     // [total_m]
    float* cf;                     // [total_m]
    float* R;                      // [total_m] column sums
};

// Dynamic shared memory of the solver: problem table, prefix sums, active flags,
// then three float vectors read as float4 (each offset a multiple of 16 bytes).
constexpr size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
struct BatchSmem {
    static constexpr size_t desc = 0;
    static constexpr size_t pref = a16(desc + sizeof(ot_problem_desc) * OT_BATCH_MAX);
    static constexpr size_t act = a16(pref + sizeof(long long) * (OT_BATCH_MAX + 1));
    static constexpr size_t gc = a16(act + sizeof(int) * OT_BATCH_MAX);
    static constexpr size_t cf = a16(gc + sizeof(float) * OT_BATCH_MAXM);
    static constexpr size_t acc = a16(cf + sizeof(float) * OT_BATCH_MAXM);
    static constexpr size_t total = a16(acc + sizeof(float) * OT_BATCH_MAXM);
};
static_assert(BatchSmem::gc % 16 == 0 && BatchSmem::cf % 16 == 0 && BatchSmem::acc % 16 == 0, "float4 alignment");
static_assert(BatchSmem::total <= 227 * 1024, "shared memory");

__device__ __forceinline__ void red_add_f32(float* p, float v) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

// Block-wide inclusive scan of OT_BATCH_MAX-bounded weights (one value per problem) into s_pref[0..count].
__device__ void batch_prefix(const BatchArgs& A, const ot_problem_desc* sd, const int* act, bool rows,
                             long long* s_pref, long long* s_wsum) {
    // each thread sums a contiguous chunk, then a warp scan of the chunk sums
    const int tid = threadIdx.x;
    const int per = (A.count + OT_BT - 1) / OT_BT;
    const int p0 = tid * per, p1 = min(A.count, p0 + per);
    long long loc = 0;
    for (int p = p0; p < p1; ++p) {
        const long long m = sd[p].m;
        loc += act[p] ? (rows ? m * m : m) : 0;
    }
    // block exclusive scan of loc
    const int lane = tid & 31, wid = tid >> 5;
    long long v = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) s_wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
        long long x = lane < OT_BW ? s_wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane < OT_BW) s_wsum[lane] = x;
    }
    __syncthreads();
    long long base = (wid > 0 ? s_wsum[wid - 1] : 0) + v - loc;
    for (int p = p0; p < p1; ++p) {
        s_pref[p] = base;
        const long long m = sd[p].m;
        base += act[p] ? (rows ? m * m : m) : 0;
    }
    if (tid == OT_BT - 1) s_pref[A.count] = base;
    __syncthreads();
}

// Largest p with s_pref[p] <= x (problems with zero weight are skipped by the caller).
__device__ __forceinline__ int find_problem(const long long* s_pref, int count, long long x) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_pref[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(OT_BT, 1) batch_solve_kernel(BatchArgs A) {
    extern __shared__ __align__(16) unsigned char dsm[];
    ot_problem_desc* sd = reinterpret_cast<ot_problem_desc*>(dsm + BatchSmem::desc);   // [count]
    long long* s_pref = reinterpret_cast<long long*>(dsm + BatchSmem::pref);            // [count+1]
    int* s_act = reinterpret_cast<int*>(dsm + BatchSmem::act);                          // [count]
    float* s_gc = reinterpret_cast<float*>(dsm + BatchSmem::gc);                        // [MAXM]
    float* s_cf = reinterpret_cast<float*>(dsm + BatchSmem::cf);                        // [MAXM]
    float* s_acc = reinterpret_cast<float*>(dsm + BatchSmem::acc);                      // [MAXM]
    __shared__ float s_red[OT_BR][OT_BW];
    __shared__ float s_rowF[OT_BR];
    __shared__ float s_rowU[OT_BR];
    __shared__ long long s_wsum[32];
    __shared__ double s_dred[OT_BW];
    __shared__ int s_flag;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int B = blockIdx.x, Gd = gridDim.x;
    const int count = A.count;
    unsigned epoch = 0;

    for (int p = tid; p < count; p += OT_BT) sd[p] = A.desc[p];
    __syncthreads();

    // ---- per-problem marginal sums and validation (problems split over blocks)
    for (int p = B; p < count; p += Gd) {
        const int m = sd[p].m;
        const long long v0 = sd[p].v_off;
        double sa = 0.0, sb = 0.0;
        int bad = 0;
        for (int i = tid; i < m; i += OT_BT) {
            const float x = A.a[v0 + i], y = A.b[v0 + i];
            bad |= !(x > 0.f && x < INFINITY) || !(y > 0.f && y < INFINITY);
            sa += x;
            sb += y;
        }
        // block sums (OT_BW warps)
        sa = warp_sum(sa);
        sb = warp_sum(sb);
        bad = __syncthreads_or(bad);
        if (lane == 0) s_dred[wid] = sa;
        __syncthreads();
        double ta = 0.0;
        for (int w2 = 0; w2 < OT_BW; ++w2) ta += s_dred[w2];
        __syncthreads();
        if (lane == 0) s_dred[wid] = sb;
        __syncthreads();
        double tb = 0.0;
        for (int w2 = 0; w2 < OT_BW; ++w2) tb += s_dred[w2];
        __syncthreads();
        if (tid == 0) {
            A.inv_sa[p] = 1.0 / ta;
            A.inv_sb[p] = 1.0 / tb;
            A.active[p] = bad ? 0 : 1;
            A.iters[p] = bad ? -1 : 0;
            A.l1acc[p] = 0.0;
            A.l1acc[count + p] = 0.0;
            A.res[p].value = 0.0;
            A.res[p].transport_cost = 0.0;
            A.res[p].marg_l1_col = 0.0;
            A.res[p].reserved[0] = 0.0;
            if (bad) {
                A.res[p].iters = 0;
                A.res[p].status = OT_ERR_ARG;
                A.res[p].marg_l1 = -1.0;
                A.res[p].marg_l2_col = -1.0;
            }
        }
        // column potentials and sums
        const float kap = (float)(1.0 / ((double)sd[p].eps * OT_LN2));
        for (int j = tid; j < m; j += OT_BT) {
            const double g0 = A.warm ? A.z_out[v0 + j] * (double)kap : 0.0;
            const float hi = (float)g0;
            A.gam[v0 + j] = g0;
            A.gc[v0 + j] = hi;
            A.cf[v0 + j] = ex2((float)(g0 - (double)hi));
            A.R[v0 + j] = 0.f;
        }
    }
    if (!grid_sync(A.ctrl, Gd, A.timeout_ns, epoch)) goto fail;

    for (int t = 1;; ++t) {
        const int cur = (t - 1) & 1, nxt = cur ^ 1;
        const long long TM = A.total_m;
        // ---------------- row phase
        for (int p = tid; p < count; p += OT_BT) s_act[p] = A.active[p];
        __syncthreads();
        batch_prefix(A, sd, s_act, true, s_pref, s_wsum);
        {
            // a row belongs to the block whose weight range holds the row's first entry
            const long long W = s_pref[count];
            const long long w0 = W * B / Gd, w1 = W * (B + 1) / Gd;
            const int pfirst = (W > 0 && w0 < w1) ? find_problem(s_pref, count, w0) : count;
            for (int p = pfirst; p < count && s_pref[p] < w1; ++p) {
                if (!s_act[p]) continue;
                const int m = sd[p].m, ld = sd[p].ld;
                const long long base = s_pref[p];
                const int r_lo = (w0 <= base) ? 0 : (int)((w0 - base + m - 1) / m);
                const int r_hi = min(m, (int)((w1 - base + m - 1) / m));
                if (r_lo >= r_hi) continue;
                const float kap = (float)(1.0 / ((double)sd[p].eps * OT_LN2));
                const long long v0 = sd[p].v_off;
                const float* Gp = A.G + sd[p].g_off;
                const double isa = A.inv_sa[p];
                // stage this problem's column potentials; clear the accumulator
                __syncthreads();
                // padded columns [m, ld): gamma = -inf, factor 0 (their entries are exactly 0)
                for (int j = tid; j < ld; j += OT_BT) {
                    const bool v = j < m;
                    s_gc[j] = v ? A.gc[v0 + j] : -INFINITY;
                    s_cf[j] = v ? A.cf[v0 + j] : 0.f;
                    s_acc[j] = 0.f;
                }
                __syncthreads();
                double l1 = 0.0;
                const int ng4 = ld >> 2;   // ld % 4 == 0; the padded cost entries are finite (0)
                for (int rb0 = r_lo; rb0 < r_hi; rb0 += OT_BR) {
                    const int nr = min(OT_BR, r_hi - rb0);
                    const bool safe = (t == 1);
                    float F[OT_BR];
#pragma unroll
                    for (int r = 0; r < OT_BR; ++r)
                        F[r] = (!safe && r < nr) ? A.fhi[cur * TM + v0 + rb0 + r] : 0.f;
                    for (int attempt = 0; attempt < 2; ++attempt) {
                        const bool shift = safe || attempt == 1;
                        if (shift) {   // explicit max shift: F_r = -max_j (gamma_j - c_rj)
                            float mx[OT_BR];
#pragma unroll
                            for (int r = 0; r < OT_BR; ++r) mx[r] = -INFINITY;
                            for (int g = tid; g < ng4; g += OT_BT) {
                                const float4 gg = reinterpret_cast<const float4*>(s_gc)[g];
#pragma unroll
                                for (int r = 0; r < OT_BR; ++r) {
                                    if (r < nr) {
                                        const float4 c = __ldg(reinterpret_cast<const float4*>(Gp + (long long)(rb0 + r) * ld) + g);
                                        mx[r] = fmaxf(mx[r], fmaxf(fmaxf(fmaf(c.x, -kap, gg.x), fmaf(c.y, -kap, gg.y)),
                                                                   fmaxf(fmaf(c.z, -kap, gg.z), fmaf(c.w, -kap, gg.w))));
                                    }
                                }
                            }
#pragma unroll
                            for (int r = 0; r < OT_BR; ++r) {
                                const float t2 = warp_max(mx[r]);
                                if (lane == 0) s_red[r][wid] = t2;
                            }
                            __syncthreads();
                            if (tid < OT_BR) {
                                float m2 = -INFINITY;
                                for (int w2 = 0; w2 < OT_BW; ++w2) m2 = fmaxf(m2, s_red[tid][w2]);
                                s_rowF[tid] = m2 > -INFINITY ? -m2 : 0.f;
                            }
                            __syncthreads();
#pragma unroll
                            for (int r = 0; r < OT_BR; ++r) F[r] = s_rowF[r];
                        }
                        // pass 1: row sums
                        float s[OT_BR];
#pragma unroll
                        for (int r = 0; r < OT_BR; ++r) s[r] = 0.f;
                        for (int g = tid; g < ng4; g += OT_BT) {
                            const float4 gg = reinterpret_cast<const float4*>(s_gc)[g];
                            const float4 cc = reinterpret_cast<const float4*>(s_cf)[g];
#pragma unroll
                            for (int r = 0; r < OT_BR; ++r) {
                                if (r < nr) {
                                    const float4 c = __ldg(reinterpret_cast<const float4*>(Gp + (long long)(rb0 + r) * ld) + g);
                                    s[r] += ex2(fmaf(c.x, -kap, gg.x) + F[r]) * cc.x + ex2(fmaf(c.y, -kap, gg.y) + F[r]) * cc.y +
                                            ex2(fmaf(c.z, -kap, gg.z) + F[r]) * cc.z + ex2(fmaf(c.w, -kap, gg.w) + F[r]) * cc.w;
                                }
                            }
                        }
#pragma unroll
                        for (int r = 0; r < OT_BR; ++r) {
                            const float t2 = warp_sum(s[r]);
                            if (lane == 0) s_red[r][wid] = t2;
                        }
                        __syncthreads();
                        if (tid == 0) s_flag = 0;
                        __syncthreads();
                        if (tid < nr) {
                            const long long gi = v0 + rb0 + tid;
                            float S = 0.f;
                            for (int w2 = 0; w2 < OT_BW; ++w2) S += s_red[tid][w2];
                            const float alpha = (float)((double)A.a[gi] * isa);
                            if (!(S > 1e-30f && S < 1e30f)) {
                                if (!shift) {
                                    l1 += fabs((double)fmaf(S, A.frf[cur * TM + gi] - 1.0f, S - alpha));
                                }
                                s_flag = 1;
                                s_rowU[tid] = 0.f;
                            } else {
                                double pnew;
                                if (!shift) {
                                    l1 += fabs((double)fmaf(S, A.frf[cur * TM + gi] - 1.0f, S - alpha));
                                    pnew = (double)F[tid] - (double)lg2(__fdividef(S, alpha));
                                } else {
                                    pnew = (double)F[tid] - (double)lg2(__fdividef(S, alpha));
                                }
                                const float hi = (float)pnew;
                                A.phi[nxt * TM + gi] = pnew;
                                A.fhi[nxt * TM + gi] = hi;
                                A.frf[nxt * TM + gi] = ex2((float)(pnew - (double)hi));
                                s_rowU[tid] = __fdividef(alpha, S);
                            }
                        }
                        if (tid >= nr && tid < OT_BR) s_rowU[tid] = 0.f;
                        __syncthreads();
                        if (!s_flag) break;
                        if (attempt == 1 && tid == 0) set_status(A.ctrl, OT_ERR_NONFINITE);
                        __syncthreads();
                    }
                    // pass 2: column contributions (second read of the band)
                    float U[OT_BR];
#pragma unroll
                    for (int r = 0; r < OT_BR; ++r) U[r] = s_rowU[r];
                    for (int g = tid; g < ng4; g += OT_BT) {
                        const float4 gg = reinterpret_cast<const float4*>(s_gc)[g];
                        const float4 cc = reinterpret_cast<const float4*>(s_cf)[g];
                        float4 ac = reinterpret_cast<float4*>(s_acc)[g];
#pragma unroll
                        for (int r = 0; r < OT_BR; ++r) {
                            if (r < nr) {
                                const float4 c = __ldg(reinterpret_cast<const float4*>(Gp + (long long)(rb0 + r) * ld) + g);
                                ac.x = fmaf(U[r], ex2(fmaf(c.x, -kap, gg.x) + F[r]) * cc.x, ac.x);
                                ac.y = fmaf(U[r], ex2(fmaf(c.y, -kap, gg.y) + F[r]) * cc.y, ac.y);
                                ac.z = fmaf(U[r], ex2(fmaf(c.z, -kap, gg.z) + F[r]) * cc.z, ac.z);
                                ac.w = fmaf(U[r], ex2(fmaf(c.w, -kap, gg.w) + F[r]) * cc.w, ac.w);
                            }
                        }
                        reinterpret_cast<float4*>(s_acc)[g] = ac;
                    }
                    __syncthreads();
                }
                // flush the segment's column contributions and L1 terms
                for (int j = tid; j < m; j += OT_BT) {
                    const float v = s_acc[j];
                    if (v != 0.f) red_add_f32(A.R + v0 + j, v);
                }
                l1 = warp_sum(l1);   // only lanes < OT_BR of warp 0 hold terms
                if (tid == 0 && l1 != 0.0) atomicAdd(A.l1acc + (size_t)(t & 1) * count + p, l1);
            }
        }
        if (!grid_sync(A.ctrl, Gd, A.timeout_ns, epoch)) goto fail;

        // ---------------- column phase
        batch_prefix(A, sd, s_act, false, s_pref, s_wsum);
        {
            const long long W = s_pref[count];
            const long long c0 = W * B / Gd, c1 = W * (B + 1) / Gd;
            for (long long cidx = c0 + tid; cidx < c1; cidx += OT_BT) {
                const int p = find_problem(s_pref, count, cidx);
                const int j = (int)(cidx - s_pref[p]);
                const long long v0 = sd[p].v_off;
                const double L1 = A.l1acc[(size_t)(t & 1) * count + p];
                const int done = t - 1;
                int st = -1;
                if (done >= 1) {
                    if (L1 != L1) st = OT_ERR_NONFINITE;
                    else if (L1 <= A.tol) st = OT_OK;
                    else if (done >= A.max_iter) st = OT_ERR_NOT_CONVERGED;
                }
                const float Rj = A.R[v0 + j];
                A.R[v0 + j] = 0.f;
                if (st >= 0) {
                    if (j == 0) {
                        A.active[p] = 0;
                        A.iters[p] = done;
                        A.res[p].iters = done;
                        A.res[p].status = st;
                        A.res[p].marg_l1 = L1;
                        A.res[p].marg_l2_col = -1.0;
                    }
                    continue;
                }
                if (j == 0) A.l1acc[(size_t)((t + 1) & 1) * count + p] = 0.0;
                if (Rj != Rj) {
                    set_status(A.ctrl, OT_ERR_NONFINITE);
                    continue;
                }
                double gnew;
                const double beta = (double)A.b[v0 + j] * A.inv_sb[p];
                if (Rj > 1e-30f && Rj < 1e30f) {
                    gnew = A.gam[v0 + j] - (double)lg2(__fdividef(Rj, (float)beta));
                } else {
                    // rare: recompute the column's log-sum-exp with an explicit max (one thread)
                    const int m = sd[p].m, ld = sd[p].ld;
                    const float kap = (float)(1.0 / ((double)sd[p].eps * OT_LN2));
                    const float* Gp = A.G + sd[p].g_off;
                    float mx = -INFINITY, s = 0.f;
                    for (int i = 0; i < m; ++i) {
                        const float x = fmaf(Gp[(long long)i * ld + j], -kap, A.fhi[nxt * TM + v0 + i]);
                        const float e = A.frf[nxt * TM + v0 + i];
                        if (x > mx) { s = fmaf(s, ex2(mx - x), e); mx = x; }
                        else s += ex2(x - mx) * e;
                    }
                    if (!(s > 0.f)) {
                        set_status(A.ctrl, OT_ERR_NONFINITE);
                        continue;
                    }
                    gnew = (double)lg2((float)beta) - (double)mx - (double)lg2(s);
                }
                const float hi = (float)gnew;
                A.gam[v0 + j] = gnew;
                A.gc[v0 + j] = hi;
                A.cf[v0 + j] = ex2((float)(gnew - (double)hi));
            }
        }
        if (!grid_sync(A.ctrl, Gd, A.timeout_ns, epoch)) goto fail;
        int any = 0;
        for (int p = tid; p < count; p += OT_BT) any |= ((volatile int*)A.active)[p];
        if (!__syncthreads_or(any)) break;
    }

    // ---------------- outputs: each block writes a share of all problems
    for (int p = B; p < count; p += Gd) {
        const int m = sd[p].m;
        const long long v0 = sd[p].v_off;
        const int it = A.iters[p];
        const int buf = it & 1;
        const double unit = (double)sd[p].eps * OT_LN2;
        const double shift = -(double)sd[p].eps * log((double)sd[p].N);
        for (int i = tid; i < m; i += OT_BT) {
            // a problem rejected by the validation gets NaN potentials
            A.w_out[v0 + i] = it < 0 ? (double)NAN : A.phi[(size_t)buf * A.total_m + v0 + i] * unit + shift;
            A.z_out[v0 + i] = it < 0 ? (double)NAN : A.gam[v0 + i] * unit;
        }
        if (tid == 0) A.res[p].reserved[1] = 4.0;   // variant code: batch
    }
    return;
fail:
    if (threadIdx.x == 0) {
        for (int p = B; p < count; p += Gd) {
            A.res[p].iters = -1;
            A.res[p].status = ld_volatile_int(&A.ctrl->status);
        }
    }
}

// ---- batched fold from points: G_p[i][j] = -eps log sum_k exp(-|x_i - R^k y_j|^2 / eps)
__global__ void __launch_bounds__(256) batch_fold_kernel(const ot_problem_desc* desc, int count,
                                                         const float2* pts, float* G_all) {
    const int p = blockIdx.y;
    if (p >= count) return;
    const ot_problem_desc d = desc[p];
    __shared__ float2 rot[256];
    for (int k = threadIdx.x; k < d.N && k < 256; k += blockDim.x) {
        float sn, cs;
        sincospif(2.0f * (float)k / (float)d.N, &sn, &cs);
        rot[k] = make_float2(cs, sn);
    }
    __syncthreads();
    const float kap = (float)(1.0 / ((double)d.eps * OT_LN2));
    const long long mm = (long long)d.m * d.ld;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < mm; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / d.ld), j = (int)(e - (long long)i * d.ld);
        if (j >= d.m) {   // row padding: a finite value (the solver gives these columns zero weight)
            G_all[d.g_off + (long long)i * d.ld + j] = 0.f;
            continue;
        }
        const float2 xi = pts[d.x_off + i], yj = pts[d.y_off + j];
        float mn = 0.f, s = 1.f;
        for (int k = 0; k < d.N; ++k) {
            const float2 r = rot[k];
            const float yx = r.x * yj.x - r.y * yj.y, yy = r.y * yj.x + r.x * yj.y;
            const float dx = xi.x - yx, dy = xi.y - yy;
            const float c = fmaf(dx, dx, dy * dy);
            if (k == 0) mn = c;
            else if (c < mn) { s = fmaf(s, ex2((c - mn) * kap), 1.0f); mn = c; }
            else s += ex2((mn - c) * kap);
        }
        G_all[d.g_off + (long long)i * d.ld + j] = mn - lg2(s) / kap;
    }
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct BatchLayout {
    size_t ctrl, desc, inv_sa, inv_sb, active, iters, l1acc, phi, fhi, frf, gam, gc, cf, R, total;
};

static BatchLayout batch_layout(int count, long long TM) {
    BatchLayout L;
    size_t o = 0;
    L.ctrl = o; o = a256(o + sizeof(Ctrl));
    L.desc = o; o = a256(o + sizeof(ot_problem_desc) * (size_t)count);
    L.inv_sa = o; o = a256(o + sizeof(double) * (size_t)count);
    L.inv_sb = o; o = a256(o + sizeof(double) * (size_t)count);
    L.active = o; o = a256(o + sizeof(int) * (size_t)count);
    L.iters = o; o = a256(o + sizeof(int) * (size_t)count);
    L.l1acc = o; o = a256(o + sizeof(double) * 2 * (size_t)count);
    L.phi = o; o = a256(o + sizeof(double) * 2 * (size_t)TM);
    L.fhi = o; o = a256(o + sizeof(float) * 2 * (size_t)TM);
    L.frf = o; o = a256(o + sizeof(float) * 2 * (size_t)TM);
    L.gam = o; o = a256(o + sizeof(double) * (size_t)TM);
    L.gc = o; o = a256(o + sizeof(float) * (size_t)TM);
    L.cf = o; o = a256(o + sizeof(float) * (size_t)TM);
    L.R = o; o = a256(o + sizeof(float) * (size_t)TM);
    L.total = o;
    return L;
}

// Host-side copy of the last prepared table (count, total_m) per workspace is not kept:
// the table header lives in the workspace itself.
struct BatchHeader {
    int count;
    int max_m;
    long long total_m;
    long long pad[6];
};

}  // namespace cyc

using namespace cyc;

extern "C" size_t ot_batch_workspace_bytes(int count, long long total_m) {
    if (count <= 0 || count > OT_BATCH_MAX || total_m <= 0) return 0;
    return a256(sizeof(BatchHeader)) + batch_layout(count, total_m).total;
}

extern "C" int ot_batch_prepare(const ot_problem_desc* descs, int count, void* workspace, size_t ws_bytes,
                                void* stream) {
    if (!descs || count <= 0 || count > OT_BATCH_MAX || !workspace) return OT_ERR_ARG;
    long long TM = 0;
    int max_m = 0;
    for (int p = 0; p < count; ++p) {
        const ot_problem_desc& d = descs[p];
        if (d.m <= 0 || d.N <= 0 || d.N > 256 || !(d.eps > 0.f) || d.ld < d.m || d.ld % 4 != 0 ||
            d.g_off % 4 != 0 || d.ld > OT_BATCH_MAXM)
            return OT_ERR_ARG;
        TM = TM > d.v_off + d.m ? TM : d.v_off + d.m;
        max_m = max_m > d.m ? max_m : d.m;
    }
    if (ws_bytes < ot_batch_workspace_bytes(count, TM) || ((uintptr_t)workspace) % 256) return OT_ERR_WORKSPACE;
    BatchHeader h;
    memset(&h, 0, sizeof(h));
    h.count = count;
    h.max_m = max_m;
    h.total_m = TM;
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)workspace;
    const BatchLayout L = batch_layout(count, TM);
    // pageable host sources: the copies are complete when cudaMemcpyAsync returns
    if (cudaMemcpyAsync(w, &h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess) return OT_ERR_CUDA;
    char* base = w + a256(sizeof(BatchHeader));
    if (cudaMemcpyAsync(base + L.desc, descs, sizeof(ot_problem_desc) * (size_t)count, cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
        return OT_ERR_CUDA;
    return OT_OK;
}

extern "C" int ot_batch_fold(int count, const float* points, float* G_all, void* workspace, size_t ws_bytes,
                             void* stream) {
    if (count <= 0 || count > OT_BATCH_MAX || !points || !G_all || !workspace) return OT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = device_sms();
    if (sms <= 0) return OT_ERR_CUDA;
    const BatchLayout L = batch_layout(count, 1);
    const ot_problem_desc* d = (const ot_problem_desc*)((char*)workspace + a256(sizeof(BatchHeader)) + L.desc);
    (void)ws_bytes;
    dim3 grid(64u, (unsigned)count);   // blocks of small problems leave early
    batch_fold_kernel<<<grid, 256, 0, st>>>(d, count, (const float2*)points, G_all);
    return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}

extern "C" int ot_batch_solve(int count, long long total_m, const float* G_all, const float* a_all,
                              const float* b_all, const ot_options* opt, double* w_all, double* z_all,
                              ot_result* results, void* workspace, size_t ws_bytes, void* stream) {
    if (count <= 0 || count > OT_BATCH_MAX || total_m <= 0 || !G_all || !a_all || !b_all || !opt || !w_all ||
        !z_all || !results || !workspace)
        return OT_ERR_ARG;
    if (opt->max_iter < 1 || opt->tol_l1 < 0.0) return OT_ERR_ARG;
    if (ws_bytes < ot_batch_workspace_bytes(count, total_m) || ((uintptr_t)workspace) % 256) return OT_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)workspace + a256(sizeof(BatchHeader));
    const BatchLayout L = batch_layout(count, total_m);
    BatchArgs A;
    memset(&A, 0, sizeof(A));
    A.count = count;
    A.total_m = total_m;
    A.G = G_all;
    A.a = a_all;
    A.b = b_all;
    A.tol = opt->tol_l1;
    A.max_iter = opt->max_iter;
    A.timeout_ns = opt->timeout_ns ? opt->timeout_ns : 10000000000ull;
    A.warm = opt->warm_start;
    A.w_out = w_all;
    A.z_out = z_all;
    A.res = results;
    A.ctrl = (Ctrl*)(base + L.ctrl);
    A.desc = (const ot_problem_desc*)(base + L.desc);
    A.inv_sa = (double*)(base + L.inv_sa);
    A.inv_sb = (double*)(base + L.inv_sb);
    A.active = (int*)(base + L.active);
    A.iters = (int*)(base + L.iters);
    A.l1acc = (double*)(base + L.l1acc);
    A.phi = (double*)(base + L.phi);
    A.fhi = (float*)(base + L.fhi);
    A.frf = (float*)(base + L.frf);
    A.gam = (double*)(base + L.gam);
    A.gc = (float*)(base + L.gc);
    A.cf = (float*)(base + L.cf);
    A.R = (float*)(base + L.R);
    if (cudaMemsetAsync(A.ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return OT_ERR_CUDA;
    const int sms = device_sms();
    if (sms <= 0) return OT_ERR_CUDA;
    const size_t smem = BatchSmem::total;
    auto kern = batch_solve_kernel;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return OT_ERR_CUDA;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, OT_BT, smem) != cudaSuccess || nb < 1)
        return OT_ERR_UNSUPPORTED;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sms);
    cfg.blockDim = dim3(OT_BT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, A) != cudaSuccess) return OT_ERR_CUDA;
    return OT_OK;
}
