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
//
// One cooperative persistent launch, three phases:
//   0. the potentials are scaled to log2 units and split once into FP32
//      (hi, lo) pairs; the marginal sums and <w, a>, <z, b> (FP64, per element);
//   1. tiles: an item is 32 rows x 256 columns, all N blocks k inside, so the
//      row and column partials accumulate over k in registers.  Warp w owns 4
//      rows, lane l the columns l + 32c (c < 8).  The cost from points is
//      |R^-k x_i - y_j|^2 (the rotation moves to the 4 rows), and the row
//      moment sum_j T y_j of block k is rotated by R^k once per row and k.
//      Per-entry arithmetic is FP32; per-row and per-column partials go to
//      FP64 accumulators by L2 atomics (FP64 bit patterns built with integer
//      operations: this GPU's FP64 pipe is slow, its L2 FP64 adds are not);
//   2. per element: marginal errors and the gradients of a, b and the points;
//      the last block to finish writes the result record.
#include "common.cuh"

namespace cyc {

int device_sms();
int run_unrolled(int m, int N, const float* a_base, const float* b_base, const float* C_base, const float* x,
                 const float* y, const float* G, float eps, int iters, ot_result* out, float* d_a, float* d_b,
                 float* d_C, float* d_x, float* d_y, void* ws, size_t ws_bytes, cudaStream_t st);
size_t unrolled_ws_bytes(int m, int N, int iters);

#define VB_THREADS 256
#define VB_WARPS (VB_THREADS / 32)
#define VB_RT 4                        // rows per warp in an item
#define VB_CT 8                        // columns per lane in an item
#define VB_ROWS (VB_WARPS * VB_RT)     // 32 rows per item
#define VB_COLS (32 * VB_CT)           // 256 columns per item

struct VArgs {
    int m, N;
    const float* a;
    const float* b;
    const double* w;
    const double* z;
    const float* C;
    const float2* x;
    const float2* y;
    double kappa;     // 1 / (eps ln 2)
    double eps;
    float* dC;
    float* d_a;
    float* d_b;
    float* d_x;
    float* d_y;
    ot_result* out;
    // workspace
    Ctrl* ctrl;
    double* rowS;     // [m]
    double* colS;     // [m]
    double* rowP;     // [m][2]  sum_jk T R^k y_j
    double* colP;     // [m][2]  sum_ik T R^-k x_i
    double* scal;     // [16]  0 sum C T, 1 sum T arg (log2 units), 2 sum a, 3 sum b, 4 <w,a>, 5 <z,b>,
                      //       6 row L1, 7 column L1, 8 column L2^2, 9 sum T
    float2* whl;      // [m]  w kappa as (hi, lo)
    float2* zhl;      // [m]  z kappa as (hi, lo)
    unsigned* done;   // blocks finished with phase 2
};

// FP32 -> the same value as an FP64 bit pattern, by integer operations (exact for normal
// values; zero and the flush-to-zero range give 0, Inf and NaN give NaN).
__device__ __forceinline__ double f2d_bits(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned b = u & 0x7fffffffu;
    const unsigned e = b >> 23;
    unsigned long long d = ((unsigned long long)b << 29) + (896ull << 52);
    d = (e == 0u) ? 0ull : d;
    d = (e == 255u) ? 0x7ff8000000000000ull : d;
    d |= (unsigned long long)(u & 0x80000000u) << 32;
    return __longlong_as_double((long long)d);
}

__device__ __forceinline__ void atomic_add_f32d(double* p, float v) {
    if (v != 0.f) atomicAdd(p, f2d_bits(v));
}

// Deterministic-order block sum of one double over VB_THREADS threads (all get the result).
__device__ __forceinline__ double vb_sum_d(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < VB_WARPS; ++w) t += red[w];
    return t;
}

// Compensated (Kahan) FP32 accumulation: s - c tracks the exact running sum.
__device__ __forceinline__ void kahan_add_f(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Sum of 16 per-lane values over the warp (transposing butterfly): lane l ends with the
// total of value (l >> 1) & 15.
__device__ __forceinline__ float warp_reduce16(float (&v)[16], int lane) {
#pragma unroll
    for (int step = 0; step < 4; ++step) {
        const int o = 16 >> step;
        const int half = 16 >> (step + 1);
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float keep = up ? v[i + half] : v[i];
            const float send = up ? v[i] : v[i + half];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <bool POINTS>
__global__ void __launch_bounds__(VB_THREADS, 1) value_kernel(VArgs A, unsigned long long timeout_ns) {
    extern __shared__ __align__(16) unsigned char vsm[];
    float2* s_rot = reinterpret_cast<float2*>(vsm);                          // [N] (cos, sin) of 2 pi k / N
    __shared__ float s_col[VB_WARPS][3][VB_COLS];
    __shared__ double s_dred[VB_WARPS];
    const int m = A.m, N = A.N;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int G = gridDim.x;
    const long long gt = (long long)blockIdx.x * VB_THREADS + tid, gs = (long long)G * VB_THREADS;
    unsigned epoch = 0;

    // ---- phase 0: (hi, lo) potentials in log2 units, marginal sums, <w, a>, <z, b>
    for (int k = tid; k < N; k += VB_THREADS) {
        float sn, cs;
        sincospif(2.0f * (float)k / (float)N, &sn, &cs);
        s_rot[k] = make_float2(cs, sn);
    }
    double sa = 0.0, sb = 0.0, wa = 0.0, zb = 0.0;
    for (long long i = gt; i < m; i += gs) {
        const double wk = A.w[i] * A.kappa, zk = A.z[i] * A.kappa;
        float h, l;
        split_f64(wk, h, l);
        A.whl[i] = make_float2(h, l);
        split_f64(zk, h, l);
        A.zhl[i] = make_float2(h, l);
        const double ai = A.a[i], bi = A.b[i];
        sa += ai;
        sb += bi;
        wa += A.w[i] * ai;
        zb += A.z[i] * bi;
    }
    sa = vb_sum_d(sa, s_dred);
    sb = vb_sum_d(sb, s_dred);
    wa = vb_sum_d(wa, s_dred);
    zb = vb_sum_d(zb, s_dred);
    if (tid == 0) {
        atomicAdd(A.scal + 2, sa);
        atomicAdd(A.scal + 3, sb);
        atomicAdd(A.scal + 4, wa);
        atomicAdd(A.scal + 5, zb);
    }
    if (!grid_sync(A.ctrl, G, timeout_ns, epoch)) {
        if (blockIdx.x == 0 && tid == 0) A.out->status = ld_volatile_int(&A.ctrl->status);
        return;
    }

    // ---- phase 1: tiles
    const int nrc = (m + VB_ROWS - 1) / VB_ROWS, ncs = (m + VB_COLS - 1) / VB_COLS;
    const long long nitems = (long long)nrc * ncs;
    const float kap = (float)A.kappa;
    const float Nf = (float)N;
    double dct = 0.0, dta = 0.0;   // per-item FP32 partials, summed in FP64
    for (long long item = blockIdx.x; item < nitems; item += G) {
        const int rc = (int)(item / ncs), csx = (int)(item % ncs);
        const int i0 = rc * VB_ROWS + wid * VB_RT;
        const int j0 = csx * VB_COLS + lane;
        // column data (constant over k)
        float zh[VB_CT], zl[VB_CT], yx[VB_CT], yy[VB_CT];
        float cS[VB_CT], cX[VB_CT], cY[VB_CT];
#pragma unroll
        for (int c = 0; c < VB_CT; ++c) {
            const int j = j0 + 32 * c;
            float2 zz = make_float2(-INFINITY, 0.f);
            float2 yv = make_float2(0.f, 0.f);
            if (j < m) {
                zz = A.zhl[j];
                if (POINTS) yv = A.y[j];
            }
            zh[c] = zz.x;
            zl[c] = zz.y;
            yx[c] = yv.x;
            yy[c] = yv.y;
            cS[c] = cX[c] = cY[c] = 0.f;
        }
        // row data
        float wh[VB_RT], wl[VB_RT], xx[VB_RT], xy[VB_RT];
        float rS[VB_RT], rX[VB_RT], rY[VB_RT];
#pragma unroll
        for (int r = 0; r < VB_RT; ++r) {
            const int i = i0 + r;
            float2 ww = make_float2(-INFINITY, 0.f);
            float2 xv = make_float2(0.f, 0.f);
            if (i < m) {
                ww = A.whl[i];
                if (POINTS) xv = A.x[i];
            }
            wh[r] = ww.x;
            wl[r] = ww.y;
            xx[r] = xv.x;
            xy[r] = xv.y;
            rS[r] = rX[r] = rY[r] = 0.f;
        }
        float crS[VB_RT];   // Kahan compensation of the row sums (over k)
#pragma unroll
        for (int r = 0; r < VB_RT; ++r) crS[r] = 0.f;
        float ict = 0.f, ita = 0.f;
        for (int k = 0; k < N; ++k) {
            const float2 rot = s_rot[k];
            float mX[VB_RT], mY[VB_RT], px[VB_RT], py[VB_RT], tk[VB_RT];
#pragma unroll
            for (int r = 0; r < VB_RT; ++r) {
                mX[r] = mY[r] = tk[r] = 0.f;
                // R^-k x_i
                px[r] = fmaf(rot.x, xx[r], rot.y * xy[r]);
                py[r] = fmaf(rot.x, xy[r], -rot.y * xx[r]);
            }
            float cst[VB_RT][VB_CT];
            if (!POINTS) {   // every stored cost of the tile in flight before any is used
                const float* Ck = A.C + (long long)k * m * m;
#pragma unroll
                for (int r = 0; r < VB_RT; ++r)
#pragma unroll
                    for (int c = 0; c < VB_CT; ++c) {
                        const int i = i0 + r, j = j0 + 32 * c;
                        cst[r][c] = (i < m && j < m) ? __ldg(Ck + (long long)i * m + j) : 0.f;
                    }
            }
            float kct = 0.f, kta = 0.f;
#pragma unroll
            for (int r = 0; r < VB_RT; ++r) {
#pragma unroll
                for (int c = 0; c < VB_CT; ++c) {
                    float cc;
                    if (POINTS) {
                        const float dx = px[r] - yx[c], dy = py[r] - yy[c];
                        cc = fmaf(dx, dx, dy * dy);
                    } else {
                        cc = cst[r][c];
                    }
                    // invalid rows / columns carry -inf potentials: T = 0
                    const float arg = fmaf(cc, -kap, wh[r] + zh[c]) + (wl[r] + zl[c]);
                    const float T = ex2(arg);
                    tk[r] += T;
                    cS[c] += T;
                    kct = fmaf(cc, T, kct);
                    kta = (T > 0.f) ? fmaf(arg, T, kta) : kta;
                    if (POINTS) {
                        mX[r] = fmaf(T, yx[c], mX[r]);
                        mY[r] = fmaf(T, yy[c], mY[r]);
                        cX[c] = fmaf(T, px[r], cX[c]);
                        cY[c] = fmaf(T, py[r], cY[c]);
                    } else if (A.dC) {
                        const int i = i0 + r, j = j0 + 32 * c;
                        if (i < m && j < m) A.dC[(long long)k * m * m + (long long)i * m + j] = Nf * T;
                    }
                }
            }
            ict += kct;
            ita += kta;
#pragma unroll
            for (int r = 0; r < VB_RT; ++r) {
                kahan_add_f(rS[r], crS[r], tk[r]);
                if (POINTS) {   // R^k (sum_j T y_j)
                    rX[r] += fmaf(rot.x, mX[r], -rot.y * mY[r]);
                    rY[r] += fmaf(rot.y, mX[r], rot.x * mY[r]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < VB_RT; ++r) rS[r] -= crS[r];
        dct += f2d_bits(ict);
        dta += f2d_bits(ita);
        // row partials: 12 values per warp reduced at once; lane 2v holds value v
        {
            float v[16];
#pragma unroll
            for (int r = 0; r < VB_RT; ++r) {
                v[3 * r] = rS[r];
                v[3 * r + 1] = rX[r];
                v[3 * r + 2] = rY[r];
            }
#pragma unroll
            for (int q = 3 * VB_RT; q < 16; ++q) v[q] = 0.f;
            const float tot = warp_reduce16(v, lane);
            const int vi = lane >> 1;
            if ((lane & 1) == 0 && vi < 3 * VB_RT) {
                const int r = vi / 3, comp = vi % 3;
                const int i = i0 + r;
                if (i < m) {
                    if (comp == 0) atomic_add_f32d(A.rowS + i, tot);
                    else if (POINTS) atomic_add_f32d(A.rowP + 2 * i + (comp - 1), tot);
                }
            }
        }
        // column partials: summed over the warps in shared memory, one set of atomics per column
#pragma unroll
        for (int c = 0; c < VB_CT; ++c) {
            s_col[wid][0][lane + 32 * c] = cS[c];
            if (POINTS) {
                s_col[wid][1][lane + 32 * c] = cX[c];
                s_col[wid][2][lane + 32 * c] = cY[c];
            }
        }
        __syncthreads();
        {
            const int j = csx * VB_COLS + tid;
            if (j < m) {
                float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
                for (int w = 0; w < VB_WARPS; ++w) {
                    s0 += s_col[w][0][tid];
                    if (POINTS) {
                        s1 += s_col[w][1][tid];
                        s2 += s_col[w][2][tid];
                    }
                }
                atomic_add_f32d(A.colS + j, s0);
                if (POINTS) {
                    atomic_add_f32d(A.colP + 2 * j, s1);
                    atomic_add_f32d(A.colP + 2 * j + 1, s2);
                }
            }
        }
        __syncthreads();
    }
    dct = vb_sum_d(dct, s_dred);
    dta = vb_sum_d(dta, s_dred);
    if (tid == 0) {
        atomicAdd(A.scal + 0, dct);
        atomicAdd(A.scal + 1, dta);
    }
    if (!grid_sync(A.ctrl, G, timeout_ns, epoch)) {
        if (blockIdx.x == 0 && tid == 0) A.out->status = ld_volatile_int(&A.ctrl->status);
        return;
    }

    // ---- phase 2: per element (FP64: a few operations per element)
    const double Sa = __ldcg(A.scal + 2), Sb = __ldcg(A.scal + 3);
    const double isa = 1.0 / Sa, isb = 1.0 / Sb;
    const double ia = isa / N, ib = isb / N;
    const double wm = __ldcg(A.scal + 4) * isa, zm = __ldcg(A.scal + 5) * isb;
    double rl1 = 0.0, cl1 = 0.0, cl2 = 0.0, tt = 0.0;
    for (long long i = gt; i < m; i += gs) {
        const double rs = __ldcg(A.rowS + i), cs = __ldcg(A.colS + i);
        rl1 += fabs(rs - (double)A.a[i] * ia);
        const double dc = cs - (double)A.b[i] * ib;
        cl1 += fabs(dc);
        cl2 += dc * dc;
        tt += rs;
        if (A.d_a) A.d_a[i] = (float)((A.w[i] - wm) * isa);
        if (A.d_b) A.d_b[i] = (float)((A.z[i] - zm) * isb);
        if (POINTS && A.d_x) {
            const float2 xi = A.x[i];
            A.d_x[2 * i] = (float)(2.0 * N * (rs * xi.x - __ldcg(A.rowP + 2 * i)));
            A.d_x[2 * i + 1] = (float)(2.0 * N * (rs * xi.y - __ldcg(A.rowP + 2 * i + 1)));
        }
        if (POINTS && A.d_y) {
            const float2 yj = A.y[i];
            A.d_y[2 * i] = (float)(2.0 * N * (cs * yj.x - __ldcg(A.colP + 2 * i)));
            A.d_y[2 * i + 1] = (float)(2.0 * N * (cs * yj.y - __ldcg(A.colP + 2 * i + 1)));
        }
    }
    rl1 = vb_sum_d(rl1, s_dred);
    cl1 = vb_sum_d(cl1, s_dred);
    cl2 = vb_sum_d(cl2, s_dred);
    tt = vb_sum_d(tt, s_dred);
    if (tid == 0) {
        atomicAdd(A.scal + 6, rl1);
        atomicAdd(A.scal + 7, cl1);
        atomicAdd(A.scal + 8, cl2);
        atomicAdd(A.scal + 9, tt);
        __threadfence();
        const unsigned ticket = atomicAdd(A.done, 1u);
        if (ticket == (unsigned)G - 1) {   // the last block: every contribution is in
            __threadfence();
            const double ct = __ldcg(A.scal + 0), ta = __ldcg(A.scal + 1);
            const double T1 = __ldcg(A.scal + 9);
            ot_result* o = A.out;
            o->transport_cost = N * ct;
            o->value = N * (ct + A.eps * OT_LN2 * ta - A.eps * T1);
            o->marg_l1 = N * __ldcg(A.scal + 6);
            o->marg_l1_col = N * __ldcg(A.scal + 7);
            o->marg_l2_col = sqrt((double)N * __ldcg(A.scal + 8));
            o->reserved[0] = N * T1;   // total plan mass
            o->status = ld_volatile_int(&A.ctrl->status) ? ld_volatile_int(&A.ctrl->status) : OT_OK;
        }
    }
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t value_ws_bytes(int m) {
    return a256(sizeof(Ctrl)) + a256(sizeof(double) * m) * 2 + a256(sizeof(double) * 2 * m) * 2 +
           a256(sizeof(double) * 16) + a256(sizeof(float2) * m) * 2 + a256(sizeof(unsigned) * 4);
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
    A.a = a_base;
    A.b = b_base;
    A.w = w;
    A.z = z;
    A.C = C_base;
    A.x = (const float2*)x;
    A.y = (const float2*)y;
    A.kappa = 1.0 / ((double)eps * OT_LN2);
    A.eps = (double)eps;
    A.dC = d_C;
    A.d_a = d_a;
    A.d_b = d_b;
    // the point gradients use the rotation of the targets; C_base wins when both are given
    A.d_x = C_base ? nullptr : d_x;
    A.d_y = C_base ? nullptr : d_y;
    A.out = out;
    A.ctrl = (Ctrl*)p; p += a256(sizeof(Ctrl));
    A.rowS = (double*)p; p += a256(sizeof(double) * m);
    A.colS = (double*)p; p += a256(sizeof(double) * m);
    A.rowP = (double*)p; p += a256(sizeof(double) * 2 * m);
    A.colP = (double*)p; p += a256(sizeof(double) * 2 * m);
    A.scal = (double*)p; p += a256(sizeof(double) * 16);
    A.whl = (float2*)p; p += a256(sizeof(float2) * m);
    A.zhl = (float2*)p; p += a256(sizeof(float2) * m);
    A.done = (unsigned*)p;
    // accumulators and control words start at zero (the split potentials are written in phase 0)
    if (cudaMemsetAsync(workspace, 0, (size_t)((char*)A.whl - (char*)workspace), st) != cudaSuccess ||
        cudaMemsetAsync(A.done, 0, sizeof(unsigned) * 4, st) != cudaSuccess)
        return OT_ERR_CUDA;
    const size_t smem = sizeof(float2) * (size_t)N;
    auto kern = C_base ? value_kernel<false> : value_kernel<true>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return OT_ERR_UNSUPPORTED;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, VB_THREADS, smem) != cudaSuccess || per_sm < 1)
        return OT_ERR_UNSUPPORTED;
    const int sms = device_sms();
    if (sms <= 0) return OT_ERR_CUDA;
    const int grid = sms * (per_sm < 2 ? per_sm : 2);
    const unsigned long long timeout_ns = 10000000000ull;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(VB_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, A, timeout_ns) != cudaSuccess) return OT_ERR_CUDA;
    return OT_OK;
}
