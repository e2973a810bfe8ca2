// C-SROT with the squared-L2 regulariser (Sec. 5.3, Theorem 2): alternating
// minimisation of the reduced dual on the GPU.
//
// Problem (Eq. problem_CROT): min sum_k <C_k, T_k> + sum phi(T_ijk) subject to
// sum_k T_k 1 = alpha, sum_k T_k^T 1 = beta (mass 1/N each), with
// phi(x) = (lam/2) x^2 for x >= 0.  Its dual (Eq. dual_problem_cyclic_ROT)
// has 2m variables; for fixed z every w_i solves
//     sum_{k,j} max(w_i + z_j - C_ijk, 0) = lam alpha_i                    (*)
// (Eq. derivative_of_objective_function = 0 with (phi*)'(y) = max(y, 0)/lam),
// and symmetrically every z_j for fixed w.  The optimal plan is
// T_ijk = max(w_i + z_j - C_ijk, 0) / lam (Eq. optimality_condition).
//
// One persistent cooperative launch, grid barriers between the phases:
//
//  row phase     block b takes rows b, b + G, ...; a row's N m terms
//                u = w_i + z_j - C_ijk are formed once and kept in registers
//                as FP32 (near the root they are small, so FP32 keeps their
//                relative precision).  They are formed from FP32 hi + lo
//                copies of the FP64 potentials: s = w_hi + z_hi with its exact
//                rounding error (TwoSum), then s - C, which is exact where it
//                matters (s within a factor 2 of C, Sterbenz), plus the small
//                parts.  The left side of (*) at u is the
//                row's marginal times lam under the current state: its L1
//                error feeds the stopping rule.  Newton's method on the convex,
//                piecewise-linear left side then finds the shift delta; it
//                stops when a step keeps the number of active terms (the root
//                lies on that linear piece).  w_i + delta is the new w_i.
//  column phase  the same over the transposed blocks for every z_j.
//
// The row phase of sweep t measures the state after sweep t-1; when its
// full-scale row L1 is <= tol that state (double-buffered w) is the output.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace cyc {

int device_sms();

#define SR_BLOCK 256
#define SR_WARPS (SR_BLOCK / 32)
#define SR_VPT_MAX 32                         // terms per thread (16 for lines of <= 4096 terms)
#define SR_MAX_ROW (SR_BLOCK * SR_VPT_MAX)    // N m <= 8192
#define SR_NEWTON_MAX 64

struct SrArgs {
    int m, N;
    const float* C;     // [N][m][m] first block row
    const float* Ct;    // [N][m][m] Ct[k][j][i] = C[k][i][j] (workspace)
    const float* a;     // [m] unnormalised
    const float* b;
    double lam;
    double tol;
    int max_iter;
    int warm;
    unsigned long long timeout_ns;
    Ctrl* ctrl;
    double* w;          // [2][m] row potentials (double-buffered)
    double* z;          // [m] column potentials
    float* wh;          // [2][m] FP32 hi and lo parts of w (split_store), for the column phase
    float* wl;
    float* zh;          // [m] the same for z, for the row phase
    float* zl;
    double* acc;        // [2] row L1 per sweep parity; [2..3] value, transport cost
    double* w_out;
    double* z_out;
    ot_result* res;
};

__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < SR_WARPS; ++q) t += red[q];
    return t;
}

__device__ __forceinline__ float block_max(float v, float* red) {
    v = warp_max(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    float t = -INFINITY;
#pragma unroll
    for (int q = 0; q < SR_WARPS; ++q) t = fmaxf(t, red[q]);
    return t;
}

// Left side of (*) at shift delta and its slope: sum of max(delta + u, 0) and
// the number of active terms.  FP32 sums (a line has few active terms, and the
// fixed reduction order gives every thread the same bits) and an exact integer
// count; both in one block reduction.
template <int VPT>
__device__ __forceinline__ void eval_side(const float (&u)[VPT], int len, float delta, float2* red, float& h,
                                          int& cnt) {
    float s = 0.f;
    int c = 0;
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
        const int idx = threadIdx.x + q * SR_BLOCK;
        const float x = delta + u[q];
        if (idx < len && x > 0.f) {
            s += x;
            ++c;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = make_float2(s, __int_as_float(c));
    __syncthreads();
    h = 0.f;
    cnt = 0;
#pragma unroll
    for (int q = 0; q < SR_WARPS; ++q) {
        const float2 r = red[q];
        h += r.x;
        cnt += __float_as_int(r.y);
    }
}

// Exact split of a potential into FP32 hi + lo (lo = the rounding error of hi).
__device__ __forceinline__ void split_store(double v, float* hi, float* lo, int i) {
    const float h = (float)v;
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
}

// One coordinate of the dual: the terms of line r (a row of C, or a row of Ct for a
// column) against the other side's potentials, solved for the shift of this line's
// potential.  Returns the shift (FP64) and the left side at zero shift.  (Potentials
// written by other blocks are read from L2: a line an SM cached in an earlier sweep
// may be stale.)
template <int VPT>
__device__ double solve_line(const float* Cl, long long kstride, int m, int N, double p_self, const float* o_hi,
                             const float* o_lo, float target, float2* red, float* red_f, float& h0) {
    const int len = N * m;
    const float a_hi = (float)p_self, a_lo = (float)(p_self - (double)a_hi);
    float u[VPT];
    float umax = -INFINITY;
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
        const int idx = threadIdx.x + q * SR_BLOCK;
        u[q] = -INFINITY;
        if (idx < len) {
            const int k = idx / m, j = idx - k * m;
            const float b_hi = __ldcg(o_hi + j), b_lo = __ldcg(o_lo + j);
            const float s = a_hi + b_hi;                          // TwoSum: s + e = a_hi + b_hi exactly
            const float bv = s - a_hi;
            const float e = (a_hi - (s - bv)) + (b_hi - bv);
            u[q] = (s - Cl[k * kstride + j]) + (e + (a_lo + b_lo));
            umax = fmaxf(umax, u[q]);
        }
    }
    float h;
    int cnt;
    eval_side(u, len, 0.f, red, h, cnt);
    h0 = h;
    float delta = 0.f;
    if (cnt == 0) {
        // no active term: start right of the root (the largest term alone reaches the target)
        delta = target - block_max(umax, red_f);
        eval_side(u, len, delta, red, h, cnt);
    }
    for (int it = 0; it < SR_NEWTON_MAX && cnt > 0; ++it) {
        const float nd = delta + (target - h) / (float)cnt;
        float h1;
        int c1;
        eval_side(u, len, nd, red, h1, c1);
        const bool same_piece = c1 == cnt;
        delta = nd;
        h = h1;
        cnt = c1;
        if (same_piece) break;
    }
    return (double)delta;
}

__global__ void __launch_bounds__(SR_BLOCK) srot_transpose_kernel(const float* __restrict__ C, float* __restrict__ Ct,
                                                                  int m, int N) {
    __shared__ float tile[32][33];
    const int k = blockIdx.z;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const float* Ck = C + (size_t)k * m * m;
    float* Ctk = Ct + (size_t)k * m * m;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        if (i < m && j < m) tile[r][threadIdx.x] = Ck[(size_t)i * m + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        if (i < m && j < m) Ctk[(size_t)j * m + i] = tile[threadIdx.x][r];
    }
}

template <int VPT>
__global__ void __launch_bounds__(SR_BLOCK) srot_kernel(SrArgs A) {
    __shared__ double s_red[SR_WARPS];
    __shared__ float2 s_red2[SR_WARPS];
    __shared__ float s_redf[SR_WARPS];
    __shared__ double s_sa, s_sb;
    const int tid = threadIdx.x;
    const int B = blockIdx.x, G = gridDim.x;
    const int m = A.m, N = A.N;
    const long long mm = (long long)m * m;
    unsigned epoch = 0;
    // marginal sums (every block, FP64) and the starting column potentials
    double sa = 0.0, sb = 0.0;
    int bad = 0;
    for (int i = tid; i < m; i += SR_BLOCK) {
        const float x = A.a[i], y = A.b[i];
        bad |= !(x > 0.f && x < INFINITY) || !(y > 0.f && y < INFINITY);
        sa += x;
        sb += y;
    }
    sa = block_sum(sa, s_red);
    sb = block_sum(sb, s_red);
    bad = __syncthreads_or(bad);
    if (tid == 0) {
        s_sa = sa;
        s_sb = sb;
    }
    __syncthreads();
    if (bad) {
        if (B == 0 && tid == 0) {
            A.res->status = OT_ERR_ARG;
            A.res->iters = 0;
            A.res->marg_l1 = -1.0;
        }
        return;
    }
    const double ia = 1.0 / (s_sa * N), ib = 1.0 / (s_sb * N);   // alpha_i = a_i ia, beta_j = b_j ib
    for (int j = B * SR_BLOCK + tid; j < m; j += G * SR_BLOCK) {
        const double z0 = A.warm ? A.z_out[j] : 0.0;
        A.z[j] = z0;
        split_store(z0, A.zh, A.zl, j);
        A.w[j] = 0.0;   // the base of the first row update (its root does not depend on it)
    }
    if (B == 0 && tid < 4) A.acc[tid] = 0.0;
    bool ok = grid_sync(A.ctrl, G, A.timeout_ns, epoch);
    int done = 0, status = OT_ERR_NOT_CONVERGED;
    double L1 = -1.0;
    int cur = 0;
    for (int t = 1; ok; ++t) {
        const int nxt = cur ^ 1;
        // ---- row phase: new w from (w_cur, z); the L1 of (w_cur, z) on the way
        double l1 = 0.0;
        for (int i = B; i < m; i += G) {
            float h0;
            const double al = (double)A.a[i] * ia;
            const double wi = __ldcg(A.w + cur * m + i);
            const double d = solve_line<VPT>(A.C + (long long)i * m, mm, m, N, wi, A.zh, A.zl, (float)(A.lam * al),
                                             s_red2, s_redf, h0);
            if (tid == 0) {
                A.w[nxt * m + i] = wi + d;
                split_store(wi + d, A.wh + nxt * m, A.wl + nxt * m, i);
                l1 += fabs((double)h0 / A.lam - al);
            }
        }
        if (tid == 0 && l1 != 0.0) atomicAdd(&A.acc[t & 1], l1);
        ok = grid_sync(A.ctrl, G, A.timeout_ns, epoch);
        if (!ok) break;
        L1 = N * ((volatile double*)A.acc)[t & 1];
        if (t > 1 && L1 != L1) {
            status = OT_ERR_NONFINITE;
            done = t - 1;
            break;
        }
        if (t > 1 && L1 <= A.tol) {
            status = OT_OK;
            done = t - 1;
            break;
        }
        if (t - 1 >= A.max_iter) {
            status = OT_ERR_NOT_CONVERGED;
            done = t - 1;
            break;
        }
        if (B == 0 && tid == 0) A.acc[(t + 1) & 1] = 0.0;   // the next sweep's accumulator (read this sweep already)
        // ---- column phase: new z from (w_nxt, z)
        for (int j = B; j < m; j += G) {
            float h0;
            const double zj = __ldcg(A.z + j);
            const double d = solve_line<VPT>(A.Ct + (long long)j * m, mm, m, N, zj, A.wh + nxt * m, A.wl + nxt * m,
                                             (float)(A.lam * (double)A.b[j] * ib), s_red2, s_redf, h0);
            if (tid == 0) {
                A.z[j] = zj + d;
                split_store(zj + d, A.zh, A.zl, j);
            }
        }
        cur = nxt;
        ok = grid_sync(A.ctrl, G, A.timeout_ns, epoch);
    }
    if (!ok) {
        if (B == 0 && tid == 0) {
            A.res->status = ld_volatile_int(&A.ctrl->status);
            A.res->iters = -1;
        }
        return;
    }
    // ---- outputs: potentials, and the primal objective of the returned state (FP64)
    double tc = 0.0, qq = 0.0;
    for (long long e = (long long)B * SR_BLOCK + tid; e < (long long)N * mm; e += (long long)G * SR_BLOCK) {
        const int k = (int)(e / mm);
        const long long r = e - k * mm;
        const int i = (int)(r / m), j = (int)(r - (long long)i * m);
        const double c = (double)A.C[e];
        const double T = fmax(__ldcg(A.w + cur * m + i) + __ldcg(A.z + j) - c, 0.0) / A.lam;
        tc += c * T;
        qq += T * T;
    }
    tc = block_sum(tc, s_red);
    qq = block_sum(qq, s_red);
    if (tid == 0) {
        atomicAdd(&A.acc[2], tc);
        atomicAdd(&A.acc[3], qq);
    }
    for (int i = B * SR_BLOCK + tid; i < m; i += G * SR_BLOCK) {
        A.w_out[i] = __ldcg(A.w + cur * m + i);
        A.z_out[i] = __ldcg(A.z + i);
    }
    if (!grid_sync(A.ctrl, G, A.timeout_ns, epoch)) return;
    if (B == 0 && tid == 0) {
        const double ctot = ((volatile double*)A.acc)[2], qtot = ((volatile double*)A.acc)[3];
        A.res->iters = done;
        A.res->status = status;
        A.res->marg_l1 = L1;
        A.res->transport_cost = N * ctot;
        A.res->value = N * (ctot + 0.5 * A.lam * qtot);
        A.res->marg_l2_col = -1.0;
        A.res->marg_l1_col = -1.0;
        A.res->reserved[0] = 0.0;
        A.res->reserved[1] = 5.0;   // variant code: C-SROT
    }
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SrLayout {
    size_t ctrl, Ct, w, z, wh, wl, zh, zl, acc, total;
};

static SrLayout sr_layout(int m, int N) {
    SrLayout L;
    size_t o = 0;
    L.ctrl = o; o = a256(o + sizeof(Ctrl));
    L.Ct = o; o = a256(o + sizeof(float) * (size_t)N * m * m);
    L.w = o; o = a256(o + sizeof(double) * 2 * (size_t)m);
    L.z = o; o = a256(o + sizeof(double) * (size_t)m);
    L.wh = o; o = a256(o + sizeof(float) * 2 * (size_t)m);
    L.wl = o; o = a256(o + sizeof(float) * 2 * (size_t)m);
    L.zh = o; o = a256(o + sizeof(float) * (size_t)m);
    L.zl = o; o = a256(o + sizeof(float) * (size_t)m);
    L.acc = o; o = a256(o + sizeof(double) * 4);
    L.total = o;
    return L;
}

}  // namespace cyc

using namespace cyc;

extern "C" size_t ot_srot_workspace_bytes(int m, int N) {
    if (m <= 0 || N <= 0 || (long long)N * m > SR_MAX_ROW) return 0;
    return sr_layout(m, N).total;
}

extern "C" int ot_srot_reduced(int m, int N, const float* a_base, const float* b_base, const float* C_base,
                               const ot_options* opt, double* w, double* z, ot_result* out, void* workspace,
                               size_t ws_bytes, void* stream) {
    if (m <= 0 || N <= 0 || !a_base || !b_base || !C_base || !opt || !w || !z || !out) return OT_ERR_ARG;
    if (!(opt->eps > 0.f) || opt->max_iter < 1 || opt->tol_l1 < 0.0) return OT_ERR_ARG;
    if ((long long)N * m > SR_MAX_ROW) return OT_ERR_UNSUPPORTED;
    const SrLayout L = sr_layout(m, N);
    if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace) % 256) return OT_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)workspace;
    SrArgs A;
    memset(&A, 0, sizeof(A));
    A.m = m;
    A.N = N;
    A.C = C_base;
    A.Ct = (const float*)(base + L.Ct);
    A.a = a_base;
    A.b = b_base;
    A.lam = (double)opt->eps;
    A.tol = opt->tol_l1;
    A.max_iter = opt->max_iter;
    A.warm = opt->warm_start;
    A.timeout_ns = opt->timeout_ns ? opt->timeout_ns : 10000000000ull;
    A.ctrl = (Ctrl*)(base + L.ctrl);
    A.w = (double*)(base + L.w);
    A.z = (double*)(base + L.z);
    A.wh = (float*)(base + L.wh);
    A.wl = (float*)(base + L.wl);
    A.zh = (float*)(base + L.zh);
    A.zl = (float*)(base + L.zl);
    A.acc = (double*)(base + L.acc);
    A.w_out = w;
    A.z_out = z;
    A.res = out;
    if (cudaMemsetAsync(A.ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return OT_ERR_CUDA;
    dim3 tg((m + 31) / 32, (m + 31) / 32, N);
    srot_transpose_kernel<<<tg, dim3(32, 8), 0, st>>>(C_base, (float*)(base + L.Ct), m, N);
    if (cudaGetLastError() != cudaSuccess) return OT_ERR_CUDA;
    const int sms = device_sms();
    if (sms <= 0) return OT_ERR_CUDA;
    // a line's terms live in registers: 16 per thread while they fit, so that more blocks share an SM
    auto kern = (long long)N * m <= SR_BLOCK * 16 ? srot_kernel<16> : srot_kernel<SR_VPT_MAX>;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, SR_BLOCK, 0) != cudaSuccess || nb < 1)
        return OT_ERR_UNSUPPORTED;
    const int grid = sms * (nb < 4 ? nb : 4);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid < m ? grid : m);
    cfg.blockDim = dim3(SR_BLOCK);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, A) == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}
