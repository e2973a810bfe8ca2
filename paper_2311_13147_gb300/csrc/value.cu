// ot_value_and_grad: objective, marginal norms and envelope gradients of the
// EROT value through the reduced problem (Theorem 2 and Sec. 5.1's 1/N
// relation); the unrolled adjoint lives in adjoint.cu.
//
// One pass over the N*m*m reduced plan entries T_ijk = exp((w_i + z_j - C_ijk)/eps):
//   transport cost  N * sum C T,   value  N * sum [C T + eps T (ln T - 1)],
//   row / column sums of S = sum_k T_k (full-scale marginal errors),
//   d_C = N T_k, and the point gradients
//   d_x_i = 2N (rowS_i x_i - sum_jk T_ijk R^k y_j),
//   d_y_j = 2N (colS_j y_j - sum_ik T_ijk R^-k x_i).
// Per-entry arithmetic is FP32 (potentials split once per tile into hi/lo);
// per-tile partials are promoted to FP64 and accumulated with FP64 atomics.
#include "common.cuh"

namespace cyc {

int device_sms();
int run_unrolled(int m, int N, const float* a_base, const float* b_base, const float* C_base, const float* x,
                 const float* y, const float* G, float eps, int iters, ot_result* out, float* d_a, float* d_b,
                 float* d_C, float* d_x, float* d_y, void* ws, size_t ws_bytes, cudaStream_t st);
size_t unrolled_ws_bytes(int m, int N, int iters);

#define VT_R 16

struct VAcc {
    double scal[4];      // sum C T, sum T * arg(log2 units), sum T, pad
};

struct VArgs {
    int m, N;
    const double* w;
    const double* z;
    const float* C;
    const float2* x;
    const float2* y;
    float kappa;
    float Nf;
    float* dC;
    double* rowS;   // [m]
    double* rowP;   // [m][2]  sum_jk T R^k y_j
    double* colS;   // [m]
    double* colP;   // [m][2]  sum_ik T R^-k x_i
    double* scal;   // [4]
};

template <bool POINTS>
__global__ void __launch_bounds__(OT_BLOCK) value_tiles(VArgs A) {
    __shared__ float s_wh[VT_R], s_wl[VT_R], s_zh[OT_BLOCK], s_zl[OT_BLOCK];
    __shared__ float s_red[OT_WARPS][VT_R][3];
    __shared__ float2 s_rot;
    __shared__ double s_dred[OT_WARPS];
    const int m = A.m, N = A.N;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int tiles_r = (m + VT_R - 1) / VT_R, tiles_c = (m + OT_BLOCK - 1) / OT_BLOCK;
    const long long ntiles = (long long)N * tiles_r * tiles_c;
    double acc_ct = 0.0, acc_ta = 0.0, acc_t = 0.0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int k = (int)(tile / ((long long)tiles_r * tiles_c));
        const int rem = (int)(tile - (long long)k * tiles_r * tiles_c);
        const int i0 = (rem / tiles_c) * VT_R, j0 = (rem % tiles_c) * OT_BLOCK;
        __syncthreads();
        if (tid < VT_R) {
            const int i = i0 + tid;
            float hi = 0.f, lo = 0.f;
            if (i < m) split_f64(A.w[i] * (double)A.kappa, hi, lo);
            s_wh[tid] = hi;
            s_wl[tid] = lo;
        }
        {
            const int j = j0 + tid;
            float hi = 0.f, lo = 0.f;
            if (j < m) split_f64(A.z[j] * (double)A.kappa, hi, lo);
            s_zh[tid] = hi;
            s_zl[tid] = lo;
        }
        if (tid == 0) {
            float sn, cs;
            sincospif(2.0f * (float)k / (float)N, &sn, &cs);
            s_rot = make_float2(cs, sn);
        }
        __syncthreads();
        const int j = j0 + tid;
        const bool jv = j < m;
        float2 ykj = make_float2(0.f, 0.f);
        if (POINTS && jv) {
            const float2 yj = A.y[j];
            ykj = make_float2(s_rot.x * yj.x - s_rot.y * yj.y, s_rot.y * yj.x + s_rot.x * yj.y);
        }
        float cs = 0.f, cx = 0.f, cy = 0.f;     // column partials over the tile rows
        float tct = 0.f, tta = 0.f, tt = 0.f;  // scalar partials
        // the tile's stored costs are loaded before any of them is used (all loads in flight)
        float cpre[VT_R];
        if (!POINTS) {
#pragma unroll
            for (int r = 0; r < VT_R; ++r)
                cpre[r] = (jv && i0 + r < m) ? __ldg(A.C + (long long)k * m * m + (long long)(i0 + r) * m + j) : 0.f;
        }
#pragma unroll
        for (int r = 0; r < VT_R; ++r) {
            const int i = i0 + r;
            float T = 0.f, rx = 0.f, ry = 0.f;
            if (jv && i < m) {
                const long long e = (long long)i * m + j;
                float cst;
                float2 xi = make_float2(0.f, 0.f);
                if (POINTS) {
                    xi = A.x[i];
                    const float dx = xi.x - ykj.x, dy = xi.y - ykj.y;
                    cst = fmaf(dx, dx, dy * dy);
                } else {
                    cst = cpre[r];
                }
                const float arg = fmaf(cst, -A.kappa, s_wh[r] + s_zh[tid]) + (s_wl[r] + s_zl[tid]);
                T = ex2(arg);
                if (A.dC) A.dC[(long long)k * m * m + e] = A.Nf * T;
                tct = fmaf(cst, T, tct);
                tta = fmaf(arg, T, tta);
                tt += T;
                cs += T;
                if (POINTS) {
                    // R^-k x_i
                    const float rxk = s_rot.x * xi.x + s_rot.y * xi.y, ryk = -s_rot.y * xi.x + s_rot.x * xi.y;
                    cx = fmaf(T, rxk, cx);
                    cy = fmaf(T, ryk, cy);
                    rx = T * ykj.x;
                    ry = T * ykj.y;
                }
            }
            // row partials over the block's columns
            float v0 = warp_sum(T), v1 = 0.f, v2 = 0.f;
            if (POINTS) { v1 = warp_sum(rx); v2 = warp_sum(ry); }
            if (lane == 0) {
                s_red[wid][r][0] = v0;
                s_red[wid][r][1] = v1;
                s_red[wid][r][2] = v2;
            }
        }
        __syncthreads();
        if (tid < VT_R * 3) {
            const int r = tid / 3, c = tid % 3;
            const int i = i0 + r;
            if (i < m && (c == 0 || POINTS)) {
                double s = 0.0;
                for (int w2 = 0; w2 < OT_WARPS; ++w2) s += (double)s_red[w2][r][c];
                if (c == 0) atomicAdd(A.rowS + i, s);
                else atomicAdd(A.rowP + 2 * i + (c - 1), s);
            }
        }
        if (jv) {
            atomicAdd(A.colS + j, (double)cs);
            if (POINTS) {
                atomicAdd(A.colP + 2 * j, (double)cx);
                atomicAdd(A.colP + 2 * j + 1, (double)cy);
            }
        }
        acc_ct += (double)tct;
        acc_ta += (double)tta;
        acc_t += (double)tt;
    }
    acc_ct = block_sum_d(acc_ct, s_dred);
    acc_ta = block_sum_d(acc_ta, s_dred);
    acc_t = block_sum_d(acc_t, s_dred);
    if (tid == 0) {
        atomicAdd(A.scal + 0, acc_ct);
        atomicAdd(A.scal + 1, acc_ta);
        atomicAdd(A.scal + 2, acc_t);
    }
}

// Finalise: values, marginal errors, marginal and point gradients (one block).
__global__ void __launch_bounds__(OT_BLOCK) value_finalize(int m, int N, const float* a, const float* b,
                                                           const double* w, const double* z, const float2* x,
                                                           const float2* y, double eps, const double* rowS,
                                                           const double* rowP, const double* colS,
                                                           const double* colP, const double* scal, ot_result* out,
                                                           float* d_a, float* d_b, float* d_x, float* d_y) {
    __shared__ double s_dred[OT_WARPS];
    const int tid = threadIdx.x;
    double sa = 0.0, sb = 0.0;
    for (int i = tid; i < m; i += OT_BLOCK) { sa += a[i]; sb += b[i]; }
    sa = block_sum_d(sa, s_dred);
    sb = block_sum_d(sb, s_dred);
    double wa = 0.0, zb = 0.0, rl1 = 0.0, cl1 = 0.0, cl2 = 0.0;
    const double ia = 1.0 / (sa * N), ib = 1.0 / (sb * N);   // one division each (FP64 divides are slow)
    for (int i = tid; i < m; i += OT_BLOCK) {
        const double al = (double)a[i] * ia, be = (double)b[i] * ib;
        wa += w[i] * a[i];
        zb += z[i] * b[i];
        rl1 += fabs(rowS[i] - al);
        const double dc = colS[i] - be;
        cl1 += fabs(dc);
        cl2 += dc * dc;
    }
    wa = block_sum_d(wa, s_dred);
    zb = block_sum_d(zb, s_dred);
    rl1 = block_sum_d(rl1, s_dred);
    cl1 = block_sum_d(cl1, s_dred);
    cl2 = block_sum_d(cl2, s_dred);
    const double isa = 1.0 / sa, isb = 1.0 / sb, wm = wa * isa, zm = zb * isb;
    for (int i = tid; i < m; i += OT_BLOCK) {
        if (d_a) d_a[i] = (float)((w[i] - wm) * isa);
        if (d_b) d_b[i] = (float)((z[i] - zm) * isb);
        if (d_x) {
            const double xs = rowS[i];
            d_x[2 * i] = (float)(2.0 * N * (xs * x[i].x - rowP[2 * i]));
            d_x[2 * i + 1] = (float)(2.0 * N * (xs * x[i].y - rowP[2 * i + 1]));
        }
        if (d_y) {
            const double ys = colS[i];
            d_y[2 * i] = (float)(2.0 * N * (ys * y[i].x - colP[2 * i]));
            d_y[2 * i + 1] = (float)(2.0 * N * (ys * y[i].y - colP[2 * i + 1]));
        }
    }
    if (tid == 0) {
        const double ct = scal[0], ta = scal[1], tt = scal[2];
        out->transport_cost = N * ct;
        out->value = N * (ct + eps * OT_LN2 * ta - eps * tt);
        out->marg_l1 = N * rl1;
        out->marg_l1_col = N * cl1;
        out->marg_l2_col = sqrt((double)N * cl2);
        out->reserved[0] = N * tt;   // total plan mass
        out->status = OT_OK;
    }
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t value_ws_bytes(int m) {
    return a256(sizeof(double) * m) * 2 + a256(sizeof(double) * 2 * m) * 2 + a256(sizeof(double) * 4);
}

}  // namespace cyc

using namespace cyc;

extern "C" int ot_value_and_grad(int m, int N, const float* a_base, const float* b_base, const float* C_base,
                                 const float* x, const float* y, const float* G, const double* w, const double* z,
                                 float eps, int adjoint, int unroll_iters, ot_result* out, float* d_a, float* d_b,
                                 float* d_C, float* d_x, float* d_y, void* workspace, size_t ws_bytes,
                                 void* stream) {
    if (m <= 0 || N <= 0 || !a_base || !b_base || !out || !(eps > 0.f)) return OT_ERR_ARG;
    if (!C_base && (!x || !y)) return OT_ERR_ARG;
    if ((d_x || d_y) && (!x || !y)) return OT_ERR_ARG;
    if (d_C && !C_base) return OT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (adjoint == OT_ADJ_UNROLLED) {
        if (!G || unroll_iters < 1) return OT_ERR_ARG;
        return run_unrolled(m, N, a_base, b_base, C_base, x, y, G, eps, unroll_iters, out, d_a, d_b, d_C, d_x, d_y,
                            workspace, ws_bytes, st);
    }
    if (adjoint != OT_ADJ_ENVELOPE || !w || !z) return OT_ERR_ARG;
    const size_t need = value_ws_bytes(m);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace) % 256) return OT_ERR_WORKSPACE;
    char* p = (char*)workspace;
    VArgs A;
    A.m = m;
    A.N = N;
    A.w = w;
    A.z = z;
    A.C = C_base;
    A.x = (const float2*)x;
    A.y = (const float2*)y;
    A.kappa = (float)(1.0 / ((double)eps * OT_LN2));
    A.Nf = (float)N;
    A.dC = d_C;
    A.rowS = (double*)p; p += a256(sizeof(double) * m);
    A.colS = (double*)p; p += a256(sizeof(double) * m);
    A.rowP = (double*)p; p += a256(sizeof(double) * 2 * m);
    A.colP = (double*)p; p += a256(sizeof(double) * 2 * m);
    A.scal = (double*)p;
    if (cudaMemsetAsync(workspace, 0, need, st) != cudaSuccess) return OT_ERR_CUDA;
    const int sms = device_sms();
    if (sms <= 0) return OT_ERR_CUDA;
    const long long ntiles = (long long)N * ((m + VT_R - 1) / VT_R) * ((m + OT_BLOCK - 1) / OT_BLOCK);
    long long grid = ntiles < (long long)sms * 4 ? ntiles : (long long)sms * 4;
    if (grid < 1) grid = 1;
    // the point gradients use the rotation of the targets; C_base wins when both are given
    if (C_base) value_tiles<false><<<(int)grid, OT_BLOCK, 0, st>>>(A);
    else value_tiles<true><<<(int)grid, OT_BLOCK, 0, st>>>(A);
    value_finalize<<<1, OT_BLOCK, 0, st>>>(m, N, a_base, b_base, w, z, (const float2*)x, (const float2*)y,
                                           (double)eps, A.rowS, A.rowP, A.colS, A.colP, A.scal, out, d_a, d_b,
                                           C_base ? nullptr : d_x, C_base ? nullptr : d_y);
    return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}
