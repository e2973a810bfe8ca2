// Unrolled-iteration adjoint of the EROT value (form 3, "unrolled" option).
//
// V_T = N(<w_T, alpha> + <z_T, beta>) - eps after T iterations of the
// log-domain cyclic Sinkhorn of Algorithm 2 from z = 0, written with the unit-
// mass marginals alpha' = a/sum(a), beta' = b/sum(b) and f' = w + eps log N:
//     V_T = <w_T, alpha'> + <z_T, beta'> - eps.
// Forward (checkpointed; phi = f'/(eps ln 2), zeta = z/(eps ln 2), g = G/(eps ln 2)):
//     f'^t_i = eps log alpha'_i - eps LSE_j((z^{t-1}_j - G_ij)/eps)
//     z^t_j  = eps log beta'_j  - eps LSE_i((f'^t_i - G_ij)/eps)
// with the row / column softmaxes
//     P^t_ij = exp((f'^t_i + z^{t-1}_j - G_ij)/eps) / alpha'_i,
//     Q^t_ij = exp((f'^t_i + z^t_j     - G_ij)/eps) / beta'_j.
// Reverse, t = T..1, adjoints fh = dV/df'^t, zh = dV/dz^t (zh^T = beta'):
//     fh^t_i     = [t = T] alpha'_i - sum_j Q^t_ij zh^t_j          (row phase)
//     zh^{t-1}_j = - sum_i P^t_ij fh^t_i                            (column phase)
//     Ghat_ij   += Q^t_ij zh^t_j + P^t_ij fh^t_i
//     ah_i      += eps fh^t_i / alpha'_i,   bh_j += eps zh^t_j / beta'_j
// then ah += w_T, bh += z_T (the direct terms), and the chains
//     d_a = (ah - <ah, alpha'>)/sum(a),  d_b likewise,
//     d_C_ijk = Ghat_ij exp((G_ij - C_ijk)/eps)        (dG_ij/dC_ijk, Eq. def_Kij)
//     d_x, d_y through C_ijk = |x_i - R^k y_j|^2.
// One cooperative launch does the forward and the reverse pass: a warp per
// row in row phases, a warp per column in column phases, a bounded grid
// barrier between phases.  Per-entry exponentials are FP32 (ex2) around FP64
// potentials split into hi/lo pairs staged in shared memory for the phase.
#include <math.h>

#include "common.cuh"

namespace cyc {

int device_sms();

struct AdjArgs {
    int m, N, T;
    const float* G;        // [m][m] folded cost
    const float* C;        // [N][m][m] blocks or null
    const float2* x;       // points or null
    const float2* y;
    const float* a;
    const float* b;
    float kappa;           // 1/(eps ln2)
    double eps;
    double unit;           // eps ln2
    ot_result* res;
    float* d_a;
    float* d_b;
    float* d_C;
    float* d_x;
    float* d_y;
    unsigned long long timeout_ns;
    // workspace
    Ctrl* ctrl;
    double* F;             // [T+1][m]  f'^t in log2 units (row 0 unused)
    double* Z;             // [T+1][m]  zeta^t (row 0 = 0)
    double* fh;            // [m]
    double* zh;            // [m]
    double* ah;            // [m]
    double* bh;            // [m]
    float* Gh;             // [m][m]
    double* red;           // [4] scalars
};

__device__ __forceinline__ void stage_hilo(const double* v, int n, float* hi, float* lo) {
    for (int i = threadIdx.x; i < n; i += OT_BLOCK) {
        const double d = v[i];
        const float h = (float)d;
        hi[i] = h;
        lo[i] = (float)(d - (double)h);
    }
}

// Online log-sum-exp of base-2 exponents: keeps (mx, s) with sum 2^(x - mx) = s.
__device__ __forceinline__ void lse_add(float& mx, float& s, float x) {
    if (x > mx) {
        s = fmaf(s, ex2(mx - x), 1.0f);
        mx = x;
    } else {
        s += ex2(x - mx);
    }
}

__device__ __forceinline__ void lse_merge(float& mx, float& s, float mx2, float s2) {
    if (mx2 > mx) {
        s = fmaf(s, ex2(mx - mx2), s2);
        mx = mx2;
    } else if (mx2 > -INFINITY) {
        s += s2 * ex2(mx2 - mx);
    }
}

__device__ __forceinline__ void warp_lse(float& mx, float& s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float m2 = __shfl_xor_sync(0xffffffffu, mx, o);
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        lse_merge(mx, s, m2, s2);
    }
}

__global__ void __launch_bounds__(OT_BLOCK, 1) unroll_kernel(AdjArgs A) {
    extern __shared__ __align__(16) float sh[];
    float* vh = sh;             // [m] hi of the staged potential
    float* vl = sh + A.m;       // [m] lo
    float* wv = sh + 2 * A.m;   // [m] staged adjoint (divided by its marginal)
    __shared__ double s_dred[OT_WARPS];
    const int m = A.m, T = A.T;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int B = blockIdx.x, Gd = gridDim.x;
    const int gw = B * OT_WARPS + wid, nw = Gd * OT_WARPS;   // global warp index / count
    unsigned epoch = 0;
    const float kap = A.kappa;

    // marginal sums (FP64, every block the same)
    double sa = 0.0, sb = 0.0;
    for (int i = tid; i < m; i += OT_BLOCK) { sa += A.a[i]; sb += A.b[i]; }
    sa = block_sum_d(sa, s_dred);
    sb = block_sum_d(sb, s_dred);
    for (int j = B * OT_BLOCK + tid; j < m; j += Gd * OT_BLOCK) {
        A.Z[j] = 0.0;
        A.ah[j] = 0.0;
        A.bh[j] = 0.0;
    }
    for (long long e = (long long)B * OT_BLOCK + tid; e < (long long)m * m; e += (long long)Gd * OT_BLOCK) A.Gh[e] = 0.f;
    if (!grid_sync(A.ctrl, Gd, A.timeout_ns, epoch)) goto fail;

    // ---------------- forward, checkpointing F[t], Z[t]
    for (int t = 1; t <= T; ++t) {
        // row phase: phi_i = log2 alpha'_i - LSE2_j(zeta_j - g_ij)
        stage_hilo(A.Z + (size_t)(t - 1) * m, m, vh, vl);
        __syncthreads();
        for (int i = gw; i < m; i += nw) {
            float mx = -INFINITY, s = 0.f;
            const float* gr = A.G + (size_t)i * m;
            for (int j = lane; j < m; j += 32) lse_add(mx, s, fmaf(__ldg(gr + j), -kap, vh[j]) + vl[j]);
            warp_lse(mx, s);
            if (lane == 0) {
                const double al = (double)A.a[i] / sa;
                A.F[(size_t)t * m + i] = (double)lg2((float)al) - (double)mx - (double)lg2(s);
            }
        }
        if (!grid_sync(A.ctrl, Gd, A.timeout_ns, epoch)) goto fail;
        // column phase: zeta_j = log2 beta'_j - LSE2_i(phi_i - g_ij)
        stage_hilo(A.F + (size_t)t * m, m, vh, vl);
        __syncthreads();
        for (int j = gw; j < m; j += nw) {
            float mx = -INFINITY, s = 0.f;
            for (int i = lane; i < m; i += 32) lse_add(mx, s, fmaf(__ldg(A.G + (size_t)i * m + j), -kap, vh[i]) + vl[i]);
            warp_lse(mx, s);
            if (lane == 0) {
                const double be = (double)A.b[j] / sb;
                A.Z[(size_t)t * m + j] = (double)lg2((float)be) - (double)mx - (double)lg2(s);
            }
        }
        if (!grid_sync(A.ctrl, Gd, A.timeout_ns, epoch)) goto fail;
    }

    // ---------------- reverse
    for (int j = B * OT_BLOCK + tid; j < m; j += Gd * OT_BLOCK) A.zh[j] = (double)A.b[j] / sb;
    if (!grid_sync(A.ctrl, Gd, A.timeout_ns, epoch)) goto fail;
    for (int t = T; t >= 1; --t) {
        // row phase: fh_i = [t = T] alpha'_i - sum_j Q_ij zh_j;  Ghat += Q * zh
        stage_hilo(A.Z + (size_t)t * m, m, vh, vl);
        for (int j = tid; j < m; j += OT_BLOCK) wv[j] = (float)(A.zh[j] / ((double)A.b[j] / sb));   // zh_j / beta'_j
        __syncthreads();
        for (int i = gw; i < m; i += nw) {
            const double fi = A.F[(size_t)t * m + i];
            const float fhi = (float)fi, flo = (float)(fi - (double)fhi);
            const float* gr = A.G + (size_t)i * m;
            float* ghr = A.Gh + (size_t)i * m;
            float acc = 0.f;
            for (int j = lane; j < m; j += 32) {
                const float q = ex2(fmaf(__ldg(gr + j), -kap, fhi + vh[j]) + (flo + vl[j]));   // Q_ij * beta'_j
                const float c = q * wv[j];                                                      // Q_ij zh_j
                acc += c;
                ghr[j] += c;
            }
            acc = warp_sum(acc);
            if (lane == 0) {
                const double al = (double)A.a[i] / sa;
                const double f = (t == T ? al : 0.0) - (double)acc;
                A.fh[i] = f;
                A.ah[i] += A.eps * f / al;
            }
        }
        if (!grid_sync(A.ctrl, Gd, A.timeout_ns, epoch)) goto fail;
        // column phase: zh^{t-1}_j = - sum_i P_ij fh_i;  Ghat += P * fh
        stage_hilo(A.F + (size_t)t * m, m, vh, vl);
        for (int i = tid; i < m; i += OT_BLOCK) wv[i] = (float)(A.fh[i] / ((double)A.a[i] / sa));   // fh_i / alpha'_i
        __syncthreads();
        for (int j = gw; j < m; j += nw) {
            const double zj = A.Z[(size_t)(t - 1) * m + j];
            const float zhi = (float)zj, zlo = (float)(zj - (double)zhi);
            float acc = 0.f;
            for (int i = lane; i < m; i += 32) {
                const size_t e = (size_t)i * m + j;
                const float p = ex2(fmaf(__ldg(A.G + e), -kap, vh[i] + zhi) + (vl[i] + zlo));   // P_ij * alpha'_i
                const float c = p * wv[i];                                                      // P_ij fh_i
                acc += c;
                A.Gh[e] += c;
            }
            acc = warp_sum(acc);
            if (lane == 0) {
                A.bh[j] += A.eps * A.zh[j] / ((double)A.b[j] / sb);
                A.zh[j] = -(double)acc;      // zh^{t-1}
            }
        }
        if (!grid_sync(A.ctrl, Gd, A.timeout_ns, epoch)) goto fail;
    }

    // ---------------- direct terms, value, marginal chains (block 0)
    if (B == 0) {
        double va = 0.0, vb = 0.0, ha = 0.0, hb = 0.0;
        for (int i = tid; i < m; i += OT_BLOCK) {
            const double al = (double)A.a[i] / sa, be = (double)A.b[i] / sb;
            const double wT = A.F[(size_t)T * m + i] * A.unit - A.eps * log((double)A.N);   // mass-1/N w_T
            const double zT = A.Z[(size_t)T * m + i] * A.unit;
            va += wT * al;
            vb += zT * be;
            const double ai = A.ah[i] + wT, bi = A.bh[i] + zT;
            A.ah[i] = ai;
            A.bh[i] = bi;
            ha += ai * al;
            hb += bi * be;
        }
        va = block_sum_d(va, s_dred);
        vb = block_sum_d(vb, s_dred);
        ha = block_sum_d(ha, s_dred);
        hb = block_sum_d(hb, s_dred);
        for (int i = tid; i < m; i += OT_BLOCK) {
            if (A.d_a) A.d_a[i] = (float)((A.ah[i] - ha) / sa);
            if (A.d_b) A.d_b[i] = (float)((A.bh[i] - hb) / sb);
        }
        if (tid == 0) {
            A.res->value = va + vb - A.eps;
            A.res->iters = T;
            A.res->status = OT_OK;
            A.res->marg_l1 = -1.0;
        }
    }
    return;
fail:
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        A.res->iters = -1;
        A.res->status = ld_volatile_int(&A.ctrl->status);
    }
}

// d_C_ijk = Ghat_ij exp((G_ij - C_ijk)/eps), or the point gradients through C_ijk = |x_i - R^k y_j|^2.
template <bool POINTS>
__global__ void __launch_bounds__(OT_BLOCK) chain_kernel(AdjArgs A) {
    __shared__ float2 s_rot[256];
    const int m = A.m, N = A.N;
    for (int k = threadIdx.x; k < N && k < 256; k += OT_BLOCK) {
        float sn, cs;
        sincospif(2.0f * (float)k / (float)N, &sn, &cs);
        s_rot[k] = make_float2(cs, sn);
    }
    __syncthreads();
    const long long mm = (long long)m * m;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < mm; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / m), j = (int)(e - (long long)i * m);
        const float gh = A.Gh[e], g = A.G[e];
        if (!POINTS) {
            for (int k = 0; k < N; ++k) {
                const float c = A.C[(long long)k * mm + e];
                A.d_C[(long long)k * mm + e] = gh * ex2((g - c) * A.kappa);
            }
        } else {
            const float2 xi = A.x[i], yj = A.y[j];
            float gx = 0.f, gy = 0.f, hx = 0.f, hy = 0.f;
            for (int k = 0; k < N; ++k) {
                const float2 r = s_rot[k];
                const float yx = r.x * yj.x - r.y * yj.y, yy = r.y * yj.x + r.x * yj.y;
                const float dx = xi.x - yx, dy = xi.y - yy;
                const float c = fmaf(dx, dx, dy * dy);
                const float w = 2.0f * gh * ex2((g - c) * A.kappa);   // dV/dC_ijk * 2
                gx += w * dx;
                gy += w * dy;
                // y_j - R^-k x_i = -R^-k (x_i - R^k y_j)
                hx -= w * (r.x * dx + r.y * dy);
                hy -= w * (-r.y * dx + r.x * dy);
            }
            if (A.d_x) { atomicAdd(A.d_x + 2 * i, gx); atomicAdd(A.d_x + 2 * i + 1, gy); }
            if (A.d_y) { atomicAdd(A.d_y + 2 * j, hx); atomicAdd(A.d_y + 2 * j + 1, hy); }
        }
    }
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct AdjLayout {
    size_t ctrl, F, Z, fh, zh, ah, bh, Gh, red, total;
};

static AdjLayout adj_layout(int m, int T) {
    AdjLayout L;
    size_t o = 0;
    L.ctrl = o; o = a256(o + sizeof(Ctrl));
    L.F = o; o = a256(o + sizeof(double) * (size_t)(T + 1) * m);
    L.Z = o; o = a256(o + sizeof(double) * (size_t)(T + 1) * m);
    L.fh = o; o = a256(o + sizeof(double) * m);
    L.zh = o; o = a256(o + sizeof(double) * m);
    L.ah = o; o = a256(o + sizeof(double) * m);
    L.bh = o; o = a256(o + sizeof(double) * m);
    L.Gh = o; o = a256(o + sizeof(float) * (size_t)m * m);
    L.red = o; o = a256(o + sizeof(double) * 4);
    L.total = o;
    return L;
}

size_t unrolled_ws_bytes(int m, int N, int iters) {
    (void)N;
    if (m <= 0 || iters < 1) return 0;
    return adj_layout(m, iters).total;
}

int run_unrolled(int m, int N, const float* a_base, const float* b_base, const float* C_base, const float* x,
                 const float* y, const float* G, float eps, int iters, ot_result* out, float* d_a, float* d_b,
                 float* d_C, float* d_x, float* d_y, void* ws, size_t ws_bytes, cudaStream_t st) {
    if ((d_x || d_y) && C_base) return OT_ERR_ARG;
    const AdjLayout L = adj_layout(m, iters);
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws) % 256) return OT_ERR_WORKSPACE;
    const size_t smem = sizeof(float) * 3 * (size_t)m;
    if (smem > 200 * 1024 || N > 256) return OT_ERR_UNSUPPORTED;
    char* w = (char*)ws;
    AdjArgs A;
    memset(&A, 0, sizeof(A));
    A.m = m;
    A.N = N;
    A.T = iters;
    A.G = G;
    A.C = C_base;
    A.x = (const float2*)x;
    A.y = (const float2*)y;
    A.a = a_base;
    A.b = b_base;
    A.kappa = (float)(1.0 / ((double)eps * OT_LN2));
    A.eps = (double)eps;
    A.unit = (double)eps * OT_LN2;
    A.res = out;
    A.d_a = d_a;
    A.d_b = d_b;
    A.d_C = d_C;
    A.d_x = d_x;
    A.d_y = d_y;
    A.timeout_ns = 10000000000ull;
    A.ctrl = (Ctrl*)(w + L.ctrl);
    A.F = (double*)(w + L.F);
    A.Z = (double*)(w + L.Z);
    A.fh = (double*)(w + L.fh);
    A.zh = (double*)(w + L.zh);
    A.ah = (double*)(w + L.ah);
    A.bh = (double*)(w + L.bh);
    A.Gh = (float*)(w + L.Gh);
    A.red = (double*)(w + L.red);
    if (cudaMemsetAsync(A.ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return OT_ERR_CUDA;
    if (d_x && cudaMemsetAsync(d_x, 0, sizeof(float) * 2 * m, st) != cudaSuccess) return OT_ERR_CUDA;
    if (d_y && cudaMemsetAsync(d_y, 0, sizeof(float) * 2 * m, st) != cudaSuccess) return OT_ERR_CUDA;
    const int sms = device_sms();
    if (sms <= 0) return OT_ERR_CUDA;
    auto kern = unroll_kernel;
    if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return OT_ERR_CUDA;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, OT_BLOCK, smem) != cudaSuccess || nb < 1)
        return OT_ERR_UNSUPPORTED;
    int grid = sms;
    const int need = (m + OT_WARPS - 1) / OT_WARPS;
    if (need < grid) grid = need;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(OT_BLOCK);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, A) != cudaSuccess) return OT_ERR_CUDA;
    if (d_C || d_x || d_y) {
        const long long mm = (long long)m * m;
        long long g2 = (mm + OT_BLOCK - 1) / OT_BLOCK;
        if (g2 > (long long)sms * 8) g2 = (long long)sms * 8;
        if (C_base) chain_kernel<false><<<(int)g2, OT_BLOCK, 0, st>>>(A);
        else chain_kernel<true><<<(int)g2, OT_BLOCK, 0, st>>>(A);
    }
    return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}

}  // namespace cyc
