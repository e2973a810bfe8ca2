// ot_fold_cost: fold the N cost blocks into the m x m reduced cost.
//
// OT_MIN    -- Theorem 1 (Eq. definition_G): G = min_k C_k, kstar = smallest argmin.
// OT_SOFTMIN-- Eq. def_Kij in log form: G = cmin - eps*log sum_k exp(-(C_k - cmin)/eps).
//
// HBM-bound streaming kernel: each thread owns 4 consecutive entries (one
// 16-byte load per block k), grid-stride over the m*m entries, grid sized to
// a multiple of the SM count.  With points instead of stored blocks the cost
// C_k[i][j] = |x_i - R^k y_j|^2 is formed in registers (no HBM traffic for C):
// column strips with the N rotated targets held in registers (N <= 16), or one
// thread per entry for larger N.
#include "common.cuh"

namespace cyc {

#define FOLD_U 8   // cost blocks loaded per round of the stored-cost folds

// min with numpy semantics: a NaN propagates and its first index is kept.
__device__ __forceinline__ void min_step(float c, int k, float& best, int& kb) {
    if (best != best) return;
    if (c != c || c < best) { best = c; kb = k; }
}

// Online soft-min: keeps s = sum_k exp2((mn - C_k) * kappa) for the running minimum mn.
__device__ __forceinline__ void softmin_step(float c, float kappa, float& mn, float& s) {
    if (c < mn) {
        s = fmaf(s, ex2((c - mn) * kappa), 1.0f);
        mn = c;
    } else {
        s += ex2((mn - c) * kappa);
    }
}

template <int MODE>
__global__ void __launch_bounds__(OT_BLOCK) fold_blocks_vec4(int N, long long mm4, const float4* __restrict__ C,
                                                             float kappa, float4* __restrict__ G,
                                                             uchar4* __restrict__ ks) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < mm4; e += stride) {
        float4 c0 = __ldg(C + e);
        float b[4] = {c0.x, c0.y, c0.z, c0.w};
        int kb[4] = {0, 0, 0, 0};
        // blocks are loaded FOLD_U at a time (all loads in flight), then folded in order of k
        float4 cks[FOLD_U];
        if (MODE == OT_MIN) {
            for (int k0 = 1; k0 < N; k0 += FOLD_U) {
#pragma unroll
                for (int u = 0; u < FOLD_U; ++u)
                    if (k0 + u < N) cks[u] = __ldg(C + (long long)(k0 + u) * mm4 + e);
#pragma unroll
                for (int u = 0; u < FOLD_U; ++u) {
                    if (k0 + u < N) {
                        min_step(cks[u].x, k0 + u, b[0], kb[0]);
                        min_step(cks[u].y, k0 + u, b[1], kb[1]);
                        min_step(cks[u].z, k0 + u, b[2], kb[2]);
                        min_step(cks[u].w, k0 + u, b[3], kb[3]);
                    }
                }
            }
            G[e] = make_float4(b[0], b[1], b[2], b[3]);
            if (ks) ks[e] = make_uchar4(kb[0], kb[1], kb[2], kb[3]);
        } else {
            // one pass, online soft-min: s = sum_k exp2((mn - C_k) * kappa) for the running minimum mn
            float s[4] = {1.f, 1.f, 1.f, 1.f};
            for (int k0 = 1; k0 < N; k0 += FOLD_U) {
#pragma unroll
                for (int u = 0; u < FOLD_U; ++u)
                    if (k0 + u < N) cks[u] = __ldg(C + (long long)(k0 + u) * mm4 + e);
#pragma unroll
                for (int u = 0; u < FOLD_U; ++u) {
                    if (k0 + u < N) {
                        softmin_step(cks[u].x, kappa, b[0], s[0]);
                        softmin_step(cks[u].y, kappa, b[1], s[1]);
                        softmin_step(cks[u].z, kappa, b[2], s[2]);
                        softmin_step(cks[u].w, kappa, b[3], s[3]);
                    }
                }
            }
            const float inv = 1.0f / kappa;
            G[e] = make_float4(b[0] - inv * lg2(s[0]), b[1] - inv * lg2(s[1]),
                               b[2] - inv * lg2(s[2]), b[3] - inv * lg2(s[3]));
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(OT_BLOCK) fold_blocks_scalar(int N, long long mm, const float* __restrict__ C,
                                                               float kappa, float* __restrict__ G,
                                                               uint8_t* __restrict__ ks) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < mm; e += stride) {
        float best = __ldg(C + e);
        int kb = 0;
        if (MODE == OT_MIN) {
            for (int k = 1; k < N; ++k) min_step(__ldg(C + (long long)k * mm + e), k, best, kb);
            G[e] = best;
            if (ks) ks[e] = (uint8_t)kb;
        } else {
            float s = 1.f;
            for (int k = 1; k < N; ++k) softmin_step(__ldg(C + (long long)k * mm + e), kappa, best, s);
            G[e] = best - lg2(s) / kappa;
        }
    }
}

// Points: C_k[i][j] = |x_i - R^k y_j|^2.  One thread per (i, j); the N
// rotations of y_j are formed from the per-block (cos, sin) table in shared memory.
template <int MODE>
__global__ void __launch_bounds__(OT_BLOCK) fold_points(int m, int N, const float2* __restrict__ x,
                                                        const float2* __restrict__ y, float kappa,
                                                        float* __restrict__ G, uint8_t* __restrict__ ks) {
    extern __shared__ float2 rot[];   // [N] (cos, sin) of 2*pi*k/N
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)k / (float)N, &s, &c);
        rot[k] = make_float2(c, s);
    }
    __syncthreads();
    const long long mm = (long long)m * m;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < mm; e += stride) {
        const int i = (int)(e / m), j = (int)(e - (long long)i * m);
        const float2 xi = __ldg(x + i), yj = __ldg(y + j);
        float best = 0.f, sum = 1.f;
        int kb = 0;
        for (int k = 0; k < N; ++k) {
            const float2 r = rot[k];
            const float yx = r.x * yj.x - r.y * yj.y, yy = r.y * yj.x + r.x * yj.y;
            const float dx = xi.x - yx, dy = xi.y - yy;
            const float c = fmaf(dx, dx, dy * dy);
            if (k == 0) best = c;
            else if (MODE == OT_MIN) min_step(c, k, best, kb);
            else softmin_step(c, kappa, best, sum);
        }
        if (MODE == OT_MIN) {
            G[e] = best;
            if (ks) ks[e] = (uint8_t)kb;
        } else {
            G[e] = best - lg2(sum) / kappa;
        }
    }
}

// Two FP32 lanes per instruction (f32x2 arithmetic, the same rounding as two scalar operations).
typedef unsigned long long fx2;
__device__ __forceinline__ fx2 fx_pk(float a, float b) {
    fx2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 fx_up(fx2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return make_float2(a, b);
}
__device__ __forceinline__ fx2 fx_sub(fx2 a, fx2 b) {
    fx2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ fx2 fx_mul(fx2 a, fx2 b) {
    fx2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ fx2 fx_fma(fx2 a, fx2 b, fx2 c) {
    fx2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ fx2 fx_add(fx2 a, fx2 b) {
    fx2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Points, column strips: a block takes 256 consecutive columns (one per thread) and a
// run of rows.  Each thread rotates its target point once per item (NK registers
// pairs), then per row forms the N costs, their minimum and, for the soft-min, the
// sum of exp2((min - C_k) kappa) in a second pass over registers (no branch).
// Stores are coalesced (a row of 256 consecutive entries per block).  N <= NK.
// The soft-min works on pairs of blocks (f32x2): the rotated targets of blocks
// k >= N sit at 1e30, so their costs are +inf, they never win the minimum and
// their exponentials are 0.
template <int MODE, int NK>
__global__ void __launch_bounds__(OT_BLOCK) fold_points_strip(int m, int N, const float2* __restrict__ x,
                                                              const float2* __restrict__ y, float kappa,
                                                              int rows_per_item, float* __restrict__ G,
                                                              uint8_t* __restrict__ ks) {
    __shared__ float2 rot[NK];   // (cos, sin) of 2 pi k / N
    if (threadIdx.x < N) {
        float s, c;
        sincospif(2.0f * (float)threadIdx.x / (float)N, &s, &c);
        rot[threadIdx.x] = make_float2(c, s);
    }
    __syncthreads();
    const int strips = (m + OT_BLOCK - 1) / OT_BLOCK;
    const int chunks = (m + rows_per_item - 1) / rows_per_item;
    const long long nitems = (long long)strips * chunks;
    const float inv = (MODE == OT_SOFTMIN) ? 1.0f / kappa : 0.f;
    for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int s = (int)(item % strips), rc = (int)(item / strips);
        const int j = s * OT_BLOCK + threadIdx.x;
        if (j >= m) continue;
        const float2 yj = __ldg(y + j);
        float yx[NK], yy[NK];
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const float2 r = rot[k < N ? k : 0];
            yx[k] = r.x * yj.x - r.y * yj.y;
            yy[k] = r.y * yj.x + r.x * yj.y;
        }
        const int i0 = rc * rows_per_item, i1 = min(m, i0 + rows_per_item);
        if constexpr (MODE == OT_SOFTMIN) {
            fx2 YX[NK / 2], YY[NK / 2];
#pragma unroll
            for (int q = 0; q < NK / 2; ++q) {
                YX[q] = fx_pk(2 * q < N ? yx[2 * q] : 1e30f, 2 * q + 1 < N ? yx[2 * q + 1] : 1e30f);
                YY[q] = fx_pk(2 * q < N ? yy[2 * q] : 1e30f, 2 * q + 1 < N ? yy[2 * q + 1] : 1e30f);
            }
            const fx2 nk = fx_pk(-kappa, -kappa);
#pragma unroll 2
            for (int i = i0; i < i1; ++i) {
                const float2 xi = __ldg(x + i);
                const fx2 X = fx_pk(xi.x, xi.x), Y = fx_pk(xi.y, xi.y);
                fx2 c[NK / 2];
                float mn = INFINITY;
#pragma unroll
                for (int q = 0; q < NK / 2; ++q) {
                    const fx2 dx = fx_sub(X, YX[q]), dy = fx_sub(Y, YY[q]);
                    c[q] = fx_fma(dx, dx, fx_mul(dy, dy));
                    const float2 cv = fx_up(c[q]);
                    mn = fminf(mn, fminf(cv.x, cv.y));
                }
                const float mk = mn * kappa;
                const fx2 mk2 = fx_pk(mk, mk);
                fx2 s2 = fx_pk(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < NK / 2; ++q) {
                    const float2 a = fx_up(fx_fma(c[q], nk, mk2));
                    s2 = fx_add(s2, fx_pk(ex2(a.x), ex2(a.y)));
                }
                const float2 sv = fx_up(s2);
                G[(long long)i * m + j] = fmaf(-inv, lg2(sv.x + sv.y), mn);
            }
            continue;
        }
#pragma unroll 2
        for (int i = i0; i < i1; ++i) {
            const float2 xi = __ldg(x + i);
            float c[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const float dx = xi.x - yx[k], dy = xi.y - yy[k];
                c[k] = fmaf(dx, dx, dy * dy);
            }
            const long long e = (long long)i * m + j;
            if (MODE == OT_MIN) {
                float best = c[0];
                int kb = 0;
#pragma unroll
                for (int k = 1; k < NK; ++k)
                    if (k < N) min_step(c[k], k, best, kb);
                G[e] = best;
                if (ks) ks[e] = (uint8_t)kb;
            } else {
                float mn = c[0];
#pragma unroll
                for (int k = 1; k < NK; ++k)
                    if (k < N) mn = fminf(mn, c[k]);
                const float mk = mn * kappa;
                float sum = 0.f;
#pragma unroll
                for (int k = 0; k < NK; ++k)
                    if (k < N) sum += ex2(fmaf(-c[k], kappa, mk));
                G[e] = fmaf(-inv, lg2(sum), mn);
            }
        }
    }
}

int grid_for(long long work, int sms) {
    long long blocks = (work + OT_BLOCK - 1) / OT_BLOCK;
    long long cap = (long long)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

int device_sms();

}  // namespace cyc

using namespace cyc;

extern "C" int ot_fold_cost(int mode, int m, int N, const float* C_base, const float* x, const float* y,
                            float eps, float* G, uint8_t* kstar, void* stream) {
    if (m <= 0 || N <= 0 || G == nullptr) return OT_ERR_ARG;
    if (mode != OT_MIN && mode != OT_SOFTMIN) return OT_ERR_ARG;
    if (mode == OT_SOFTMIN && !(eps > 0.f)) return OT_ERR_ARG;
    if (C_base == nullptr && (x == nullptr || y == nullptr)) return OT_ERR_ARG;
    if (mode == OT_MIN && N > 255) return OT_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const float kappa = mode == OT_SOFTMIN ? (float)(1.0 / ((double)eps * OT_LN2)) : 0.f;
    const long long mm = (long long)m * m;
    const int sms = device_sms();
    if (sms <= 0) return OT_ERR_CUDA;
    if (C_base) {
        const bool vec = (mm % 4 == 0) && (((uintptr_t)C_base | (uintptr_t)G) % 16 == 0) &&
                         (kstar == nullptr || ((uintptr_t)kstar % 4 == 0));
        if (vec) {
            const int grid = grid_for(mm / 4, sms);
            if (mode == OT_MIN)
                fold_blocks_vec4<OT_MIN><<<grid, OT_BLOCK, 0, st>>>(N, mm / 4, (const float4*)C_base, kappa,
                                                                    (float4*)G, (uchar4*)kstar);
            else
                fold_blocks_vec4<OT_SOFTMIN><<<grid, OT_BLOCK, 0, st>>>(N, mm / 4, (const float4*)C_base, kappa,
                                                                        (float4*)G, (uchar4*)kstar);
        } else {
            const int grid = grid_for(mm, sms);
            if (mode == OT_MIN)
                fold_blocks_scalar<OT_MIN><<<grid, OT_BLOCK, 0, st>>>(N, mm, C_base, kappa, G, kstar);
            else
                fold_blocks_scalar<OT_SOFTMIN><<<grid, OT_BLOCK, 0, st>>>(N, mm, C_base, kappa, G, kstar);
        }
    } else if (N <= 16) {
        // column strips x runs of rows: about 4 items per SM
        const int strips = (m + OT_BLOCK - 1) / OT_BLOCK;
        int rpi = (int)(((long long)m * strips + 4LL * sms - 1) / (4LL * sms));
        if (rpi < 16) rpi = 16;
        const long long items = (long long)strips * ((m + rpi - 1) / rpi);
        const int grid = (int)(items < 4LL * sms ? items : 4LL * sms);
        auto launch = [&](auto kern) { kern<<<grid, OT_BLOCK, 0, st>>>(m, N, (const float2*)x, (const float2*)y, kappa,
                                                                      rpi, G, kstar); };
        if (mode == OT_MIN) {
            if (N <= 4) launch(fold_points_strip<OT_MIN, 4>);
            else if (N <= 8) launch(fold_points_strip<OT_MIN, 8>);
            else launch(fold_points_strip<OT_MIN, 16>);
        } else {
            if (N <= 4) launch(fold_points_strip<OT_SOFTMIN, 4>);
            else if (N <= 8) launch(fold_points_strip<OT_SOFTMIN, 8>);
            else launch(fold_points_strip<OT_SOFTMIN, 16>);
        }
    } else {
        const int grid = grid_for(mm, sms);
        const size_t shm = sizeof(float2) * (size_t)N;
        if (mode == OT_MIN)
            fold_points<OT_MIN><<<grid, OT_BLOCK, shm, st>>>(m, N, (const float2*)x, (const float2*)y, kappa, G,
                                                             kstar);
        else
            fold_points<OT_SOFTMIN><<<grid, OT_BLOCK, shm, st>>>(m, N, (const float2*)x, (const float2*)y, kappa,
                                                                 G, kstar);
    }
    return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}
