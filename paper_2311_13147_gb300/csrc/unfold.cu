// ot_unfold_plan: reconstruct the block-circulant plan from the reduced solution.
//
// LOT  (Theorem 1, Eq. optimal_solution_problem_CLOT): T_k[i][j] = S[i][j] if k == kstar[i][j] else 0.
// EROT (Algorithm 2's reconstruction, Theorem 2 Eq. optimality_condition):
//      T_k[i][j] = exp((w_i + z_j - C_k[i][j]) / eps).
// Layout: compact first block row [N][m][m], or the dense n x n matrix with
// T[r*m+i][c*m+j] = T_{(c-r) mod N}[i][j] (Lemma 1).
//
// Write-bound kernel.  A block covers a tile of TR rows x TC columns of one
// block T_k; the potentials of the tile are split once into FP32 hi/lo pairs
// in shared memory, so the per-entry work is FP32: 2^((wh_i + zh_j) - c_ij + (wl_i + zl_j)).
// In dense mode each computed tile is stored N times (the N positions of
// block k in the circulant), so every exponential is computed once.
#include "common.cuh"

namespace cyc {

int device_sms();

#define UT_R 16
#define UT_C 256

template <int MODE, bool POINTS>
__global__ void __launch_bounds__(OT_BLOCK) unfold_kernel(int m, int N, const float* __restrict__ S,
                                                          const double* __restrict__ w, const double* __restrict__ z,
                                                          const float* __restrict__ C, const float2* __restrict__ x,
                                                          const float2* __restrict__ y,
                                                          const uint8_t* __restrict__ ks, float kappa, int dense,
                                                          float* __restrict__ T) {
    __shared__ float s_wh[UT_R], s_wl[UT_R], s_zh[UT_C], s_zl[UT_C];
    __shared__ float2 s_rot;
    const int tiles_r = (m + UT_R - 1) / UT_R, tiles_c = (m + UT_C - 1) / UT_C;
    const long long ntiles = (long long)N * tiles_r * tiles_c;
    const long long n = (long long)N * m;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int k = (int)(tile / ((long long)tiles_r * tiles_c));
        const int rem = (int)(tile - (long long)k * tiles_r * tiles_c);
        const int i0 = (rem / tiles_c) * UT_R, j0 = (rem % tiles_c) * UT_C;
        __syncthreads();
        if (MODE == OT_PLAN_EROT) {
            if (threadIdx.x < UT_R) {
                const int i = i0 + threadIdx.x;
                float hi = 0.f, lo = 0.f;
                if (i < m) split_f64(w[i] * (double)kappa, hi, lo);
                s_wh[threadIdx.x] = hi;
                s_wl[threadIdx.x] = lo;
            }
            for (int c = threadIdx.x; c < UT_C; c += OT_BLOCK) {
                const int j = j0 + c;
                float hi = 0.f, lo = 0.f;
                if (j < m) split_f64(z[j] * (double)kappa, hi, lo);
                s_zh[c] = hi;
                s_zl[c] = lo;
            }
            if (POINTS && threadIdx.x == 0) {
                float sn, cs;
                sincospif(2.0f * (float)k / (float)N, &sn, &cs);
                s_rot = make_float2(cs, sn);
            }
        }
        __syncthreads();
        const int c = threadIdx.x;   // one column per thread, UT_C == OT_BLOCK
        const int j = j0 + c;
        if (j >= m) continue;
        float2 ykj = make_float2(0.f, 0.f);
        if (POINTS) {
            const float2 yj = y[j];
            ykj = make_float2(s_rot.x * yj.x - s_rot.y * yj.y, s_rot.y * yj.x + s_rot.x * yj.y);
        }
        for (int r = 0; r < UT_R; ++r) {
            const int i = i0 + r;
            if (i >= m) break;
            const long long e = (long long)i * m + j;
            float v;
            if (MODE == OT_PLAN_LOT) {
                v = (ks[e] == k) ? S[e] : 0.f;
            } else {
                float cst;
                if (POINTS) {
                    const float2 xi = x[i];
                    const float dx = xi.x - ykj.x, dy = xi.y - ykj.y;
                    cst = fmaf(dx, dx, dy * dy);
                } else {
                    cst = __ldg(C + (long long)k * m * m + e);
                }
                const float arg = fmaf(cst, -kappa, s_wh[r] + s_zh[c]) + (s_wl[r] + s_zl[c]);
                v = ex2(arg);
            }
            if (!dense) {
                T[(long long)k * m * m + e] = v;
            } else {
                // block (rb, cb) with (cb - rb) mod N == k
                for (int rb = 0; rb < N; ++rb) {
                    const int cb = (rb + k) % N;
                    T[((long long)rb * m + i) * n + (long long)cb * m + j] = v;
                }
            }
        }
    }
}

// EROT unfold, 4 consecutive columns per thread (m % 4 == 0, 16-byte aligned
// buffers).  An item is one block k, a strip of 1024 columns and a run of at most
// UT_RMAX rows: the strip's column potentials and the run's row potentials are
// split into (hi, lo) once per item (the FP64 work of this GPU is slow; one
// barrier per item), then sub-tiles of UT_R rows are formed with the tile's cost
// rows (or points) loaded before any exponential, two entries per f32x2
// instruction, stores with the streaming hint.
#define UT_C4 (4 * OT_BLOCK)
#define UT_RMAX 1024
typedef unsigned long long ux2;
__device__ __forceinline__ ux2 ux_pk(float a, float b) {
    ux2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 ux_up(ux2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return make_float2(a, b);
}
__device__ __forceinline__ ux2 ux_add(ux2 a, ux2 b) {
    ux2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ ux2 ux_sub(ux2 a, ux2 b) {
    ux2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ ux2 ux_mul(ux2 a, ux2 b) {
    ux2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ ux2 ux_fma(ux2 a, ux2 b, ux2 c) {
    ux2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

template <bool POINTS>
__global__ void __launch_bounds__(OT_BLOCK) unfold_erot_vec4(int m, int N, const double* __restrict__ w,
                                                             const double* __restrict__ z,
                                                             const float* __restrict__ C, const float2* __restrict__ x,
                                                             const float2* __restrict__ y, float kappa, int dense,
                                                             int rows_per_item, float* __restrict__ T) {
    __shared__ float2 s_w[UT_RMAX];   // the run's row potentials (hi, lo)
    __shared__ float4 s_zh[OT_BLOCK], s_zl[OT_BLOCK];
    __shared__ float2 s_rot;
    const int strips = (m + UT_C4 - 1) / UT_C4, chunks = (m + rows_per_item - 1) / rows_per_item;
    const long long nitems = (long long)N * strips * chunks;
    const long long n = (long long)N * m;
    const int m4 = m >> 2;
    const ux2 nk = ux_pk(-kappa, -kappa);
    for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int k = (int)(item / ((long long)strips * chunks));
        const int rem = (int)(item - (long long)k * strips * chunks);
        const int r_beg = (rem / strips) * rows_per_item, g0 = (rem % strips) * OT_BLOCK;   // float4 column index
        const int r_end = min(m, r_beg + rows_per_item);
        __syncthreads();   // the previous item's potentials are no longer read
        {
            const int g = g0 + threadIdx.x;
            float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
            if (g < m4) {
#pragma unroll
                for (int c = 0; c < 4; ++c) split_f64(z[4 * g + c] * (double)kappa, h[c], l[c]);
            }
            s_zh[threadIdx.x] = make_float4(h[0], h[1], h[2], h[3]);
            s_zl[threadIdx.x] = make_float4(l[0], l[1], l[2], l[3]);
        }
        for (int t = threadIdx.x; t < r_end - r_beg; t += OT_BLOCK) {
            float hi, lo;
            split_f64(w[r_beg + t] * (double)kappa, hi, lo);
            s_w[t] = make_float2(hi, lo);
        }
        if (POINTS && threadIdx.x == 0) {
            float sn, cs;
            sincospif(2.0f * (float)k / (float)N, &sn, &cs);
            s_rot = make_float2(cs, sn);
        }
        __syncthreads();
        const int g = g0 + threadIdx.x;
        if (g >= m4) continue;
        const float4 zh = s_zh[threadIdx.x], zl = s_zl[threadIdx.x];
        const ux2 ZH01 = ux_pk(zh.x, zh.y), ZH23 = ux_pk(zh.z, zh.w), ZL01 = ux_pk(zl.x, zl.y), ZL23 = ux_pk(zl.z, zl.w);
        ux2 YX01 = 0, YX23 = 0, YY01 = 0, YY23 = 0;
        if (POINTS) {
            float2 yk[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float2 yj = y[4 * g + c];
                yk[c] = make_float2(s_rot.x * yj.x - s_rot.y * yj.y, s_rot.y * yj.x + s_rot.x * yj.y);
            }
            YX01 = ux_pk(yk[0].x, yk[1].x);
            YX23 = ux_pk(yk[2].x, yk[3].x);
            YY01 = ux_pk(yk[0].y, yk[1].y);
            YY23 = ux_pk(yk[2].y, yk[3].y);
        }
        for (int i0 = r_beg; i0 < r_end; i0 += UT_R) {
            const int nr = min(UT_R, r_end - i0);
            ux2 c01[UT_R], c23[UT_R];
#pragma unroll
            for (int r = 0; r < UT_R; ++r) {
                if (r < nr) {
                    const int i = i0 + r;
                    if (POINTS) {
                        const float2 xi = x[i];
                        const ux2 X = ux_pk(xi.x, xi.x), Y = ux_pk(xi.y, xi.y);
                        ux2 dx = ux_sub(X, YX01), dy = ux_sub(Y, YY01);
                        c01[r] = ux_fma(dx, dx, ux_mul(dy, dy));
                        dx = ux_sub(X, YX23);
                        dy = ux_sub(Y, YY23);
                        c23[r] = ux_fma(dx, dx, ux_mul(dy, dy));
                    } else {
                        const float4 cv = __ldg(reinterpret_cast<const float4*>(C + (long long)k * m * m + (long long)i * m) + g);
                        c01[r] = ux_pk(cv.x, cv.y);
                        c23[r] = ux_pk(cv.z, cv.w);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < UT_R; ++r) {
                if (r < nr) {
                    const int i = i0 + r;
                    const float2 wv = s_w[i - r_beg];
                    const ux2 WH = ux_pk(wv.x, wv.x), WL = ux_pk(wv.y, wv.y);
                    // 2^(hi + lo - kappa c): the same operations, in the same order, as one lane at a time
                    const float2 a01 = ux_up(ux_add(ux_fma(c01[r], nk, ux_add(WH, ZH01)), ux_add(WL, ZL01)));
                    const float2 a23 = ux_up(ux_add(ux_fma(c23[r], nk, ux_add(WH, ZH23)), ux_add(WL, ZL23)));
                    const float4 v = make_float4(ex2(a01.x), ex2(a01.y), ex2(a23.x), ex2(a23.y));
                    if (!dense) {
                        __stcs(reinterpret_cast<float4*>(T + (long long)k * m * m + (long long)i * m) + g, v);
                    } else {
                        for (int rb = 0; rb < N; ++rb) {
                            const int cb = (rb + k) % N;
                            __stcs(reinterpret_cast<float4*>(T + ((long long)rb * m + i) * n + (long long)cb * m) + g, v);
                        }
                    }
                }
            }
        }
    }
}

}  // namespace cyc

using namespace cyc;

extern "C" int ot_unfold_plan(int mode, int m, int N, const void* S_or_w, const double* z, const float* C_base,
                              const float* x, const float* y, const uint8_t* kstar, float eps, int dense, float* T,
                              void* stream) {
    if (m <= 0 || N <= 0 || !S_or_w || !T) return OT_ERR_ARG;
    if (mode == OT_PLAN_LOT) {
        if (!kstar || N > 255) return OT_ERR_ARG;
    } else if (mode == OT_PLAN_EROT) {
        if (!z || !(eps > 0.f)) return OT_ERR_ARG;
        if (!C_base && (!x || !y)) return OT_ERR_ARG;
    } else {
        return OT_ERR_ARG;
    }
    const int sms = device_sms();
    if (sms <= 0) return OT_ERR_CUDA;
    const long long ntiles = (long long)N * ((m + UT_R - 1) / UT_R) * ((m + UT_C - 1) / UT_C);
    long long grid = ntiles < (long long)sms * 8 ? ntiles : (long long)sms * 8;
    if (grid < 1) grid = 1;
    const float kappa = mode == OT_PLAN_EROT ? (float)(1.0 / ((double)eps * OT_LN2)) : 0.f;
    cudaStream_t st = (cudaStream_t)stream;
    if (mode == OT_PLAN_LOT)
        unfold_kernel<OT_PLAN_LOT, false><<<(int)grid, OT_BLOCK, 0, st>>>(
            m, N, (const float*)S_or_w, nullptr, nullptr, nullptr, nullptr, nullptr, kstar, 0.f, dense, T);
    else if (m % 4 == 0 && ((uintptr_t)T) % 16 == 0 && (!C_base || ((uintptr_t)C_base) % 16 == 0)) {
        // runs of rows sized for about 8 items per SM (at least one sub-tile)
        const long long strips = (m + UT_C4 - 1) / UT_C4;
        long long rpi = ((long long)N * strips * m + 8LL * sms - 1) / (8LL * sms);
        rpi = (rpi + UT_R - 1) / UT_R * UT_R;
        if (rpi < UT_R) rpi = UT_R;
        if (rpi > UT_RMAX) rpi = UT_RMAX;   // the run's row potentials fit the block's table
        const long long nt4 = (long long)N * strips * ((m + rpi - 1) / rpi);
        const int g4 = (int)(nt4 < (long long)sms * 8 ? nt4 : (long long)sms * 8);
        if (C_base)
            unfold_erot_vec4<false><<<g4, OT_BLOCK, 0, st>>>(m, N, (const double*)S_or_w, z, C_base, nullptr, nullptr,
                                                            kappa, dense, (int)rpi, T);
        else
            unfold_erot_vec4<true><<<g4, OT_BLOCK, 0, st>>>(m, N, (const double*)S_or_w, z, nullptr,
                                                           (const float2*)x, (const float2*)y, kappa, dense,
                                                           (int)rpi, T);
    } else if (C_base)
        unfold_kernel<OT_PLAN_EROT, false><<<(int)grid, OT_BLOCK, 0, st>>>(
            m, N, nullptr, (const double*)S_or_w, z, C_base, nullptr, nullptr, nullptr, kappa, dense, T);
    else
        unfold_kernel<OT_PLAN_EROT, true><<<(int)grid, OT_BLOCK, 0, st>>>(
            m, N, nullptr, (const double*)S_or_w, z, nullptr, (const float2*)x, (const float2*)y, nullptr, kappa,
            dense, T);
    return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}
