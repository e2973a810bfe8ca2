// Kernel-domain Sinkhorn on 64 right-hand sides sharing one folded cost, with
// the two matrix products of every iteration on the tcgen05 tensor cores.
//
// Algorithm 2 written in scaling form (the closed forms of Eq.
// optimal_f_sinkhorn_logdomain exponentiated): with K = exp(-G^eps / eps) and
// marginals alpha_n, beta_n of unit mass, one iteration is
//     U = alpha ./ (K V),    V = beta ./ (K^T U)
// for all 64 histogram pairs n at once, i.e. two [m x m] x [m x 64] products.
// K and K^T are stored as BF16 (padded to mp, a multiple of 128), the products
// accumulate in FP32 in tensor memory.  BF16 limits the fixed point's accuracy
// to about 1e-3; the FP32 log-domain batch solver then polishes each pair from
// z = eps log V (warm start) to the requested tolerance.
//
// GEMM kernel (one 128-row tile of the output and one slice of the reduction
// per CTA, 128 threads):
//   thread 0      TMA producer: K tile [128 x 64] and scaling tile [64 x 64]
//                 per 64-wide reduction block into a 4-stage ring (128-byte
//                 swizzle), completion counted on the stage's mbarrier;
//   thread 32     MMA issuer: 4 tcgen05.mma (M 128, N 64, K 16, BF16 -> FP32)
//                 per stage, then tcgen05.commit frees the stage;
//   all 4 warps   epilogue: tcgen05.ld of the 128 x 64 FP32 accumulator (warp w
//                 reads lanes 32w..32w+31), stored as this reduction slice's
//                 partial product [64][mp] (one row per right-hand side); the
//                 scaling update sums the slices.
// Every wait is bounded; an expired wait sets an error flag and the CTA still
// frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace cyc {

int device_sms();

#define KD_BM 128                  // output rows per CTA (MMA M)
#define KD_BN 64                   // right-hand sides (MMA N)
#define KD_BK 64                   // reduction block per stage (one 128-byte swizzle row of BF16)
#define KD_STAGES 4
#define KD_A_BYTES (KD_BM * KD_BK * 2)
#define KD_B_BYTES (KD_BN * KD_BK * 2)
#define KD_STAGE_BYTES (KD_A_BYTES + KD_B_BYTES)
#define KD_SMEM (KD_STAGES * KD_STAGE_BYTES + 1024)
#define KD_MAX_SPLITS 16           // reduction slices (each stores its own partial product)

// ---- tcgen05 / TMA helpers (inline PTX)

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_addr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(unsigned* slot, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void umma_bf16(unsigned d_tmem, unsigned long long a_desc, unsigned long long b_desc,
                                          unsigned idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// start address >> 4 in bits [0,14), leading byte offset (unused for this
// layout) in [16,30), stride byte offset 1024 (8 rows x 128 B) >> 4 in
// [32,46), descriptor version 1 in [46,48), swizzle mode 2 (128 B) in [61,64).
__device__ __forceinline__ unsigned long long smem_desc_sw128(const void* tile) {
    const unsigned long long addr = smem_addr(tile);
    return ((addr >> 4) & 0x3FFFull) | (1ull << 16) | ((1024ull >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits [4,6) = 1), A and B
// BF16 (bits [7,10) and [10,13) = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits [17,23), M >> 4 in bits [24,29).
#define KD_IDESC ((1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(KD_BN >> 3) << 17) | ((unsigned)(KD_BM >> 4) << 24))

struct GemmArgs {
    int mp;                       // padded size (multiple of 128)
    int kb_per_split;             // reduction blocks (of 64) per CTA slice
    float* Dp;                    // [splits][64][mp] partial products, one slice per blockIdx.y
    int* err;                     // error flag (OT_ERR_TIMEOUT on an expired wait)
    unsigned long long timeout_ns;
};

// Dp[s][n][i] = sum over slice s of k of A[i][k] X[n][k] for this CTA's rows i.
// A: tensor map of a [mp][mp] BF16 matrix (row-major, K-major operand);
// X: tensor map of the [64][mp] BF16 scaling vectors (K-major operand).
__global__ void __launch_bounds__(128, 1) kd_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmX, GemmArgs g) {
    extern __shared__ unsigned char kd_smem_raw[];
    __shared__ __align__(8) unsigned long long full[KD_STAGES], empty[KD_STAGES], accb;
    __shared__ unsigned tmem_slot;
    __shared__ int s_issued;
    unsigned char* base =
        (unsigned char*)(((uintptr_t)kd_smem_raw + 1023) & ~(uintptr_t)1023);   // 1024-byte aligned tiles
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * KD_BM;
    const int nkb_total = g.mp / KD_BK;
    const int kb0 = blockIdx.y * g.kb_per_split;
    const int kb1 = min(nkb_total, kb0 + g.kb_per_split);
    const int nkb = kb1 - kb0;   // >= 1 (the host sizes the split)

    if (tid == 0) {
        for (int s = 0; s < KD_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accb, 1);
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(&tmem_slot, KD_BN);   // 64 FP32 columns x 128 lanes
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer
        int i = 0;
        for (; i < nkb; ++i) {
            const int s = i % KD_STAGES;
            const unsigned ph = (unsigned)((i / KD_STAGES) & 1);
            if (!mbar_wait(&empty[s], ph ^ 1u, g.timeout_ns)) {
                atomicExch(g.err, OT_ERR_TIMEOUT);
                break;
            }
            unsigned char* st = base + (size_t)s * KD_STAGE_BYTES;
            mbar_arrive_expect_tx(&full[s], KD_STAGE_BYTES);
            const int kc = (kb0 + i) * KD_BK;
            tma_load_2d(st, &tmA, kc, m0, &full[s]);
            tma_load_2d(st + KD_A_BYTES, &tmX, kc, 0, &full[s]);
        }
        s_issued = i;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const unsigned idesc = KD_IDESC;
        for (int i = 0; i < nkb; ++i) {
            const int s = i % KD_STAGES;
            const unsigned ph = (unsigned)((i / KD_STAGES) & 1);
            if (!mbar_wait(&full[s], ph, g.timeout_ns)) {
                atomicExch(g.err, OT_ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            unsigned char* st = base + (size_t)s * KD_STAGE_BYTES;
            const unsigned long long da = smem_desc_sw128(st), db = smem_desc_sw128(st + KD_A_BYTES);
#pragma unroll
            for (int kk = 0; kk < KD_BK / 16; ++kk) {
                // the K step of 16 BF16 = 32 bytes advances the start address inside the swizzle row
                umma_bf16(tmem, da + (unsigned long long)(2 * kk), db + (unsigned long long)(2 * kk), idesc,
                          (i > 0 || kk > 0) ? 1 : 0);
            }
            umma_commit(&empty[s]);   // the stage is free once these MMAs have read it
        }
        umma_commit(&accb);           // the accumulator is complete
    }
    __syncwarp();

    // epilogue: 128 rows x 64 columns from tensor memory
    const bool ok = mbar_wait(&accb, 0u, g.timeout_ns);
    if (!ok && lane == 0) atomicExch(g.err, OT_ERR_TIMEOUT);
    tc_fence_after();
    if (__all_sync(0xffffffffu, ok)) {
        const int row = m0 + 32 * warp + lane;
        const unsigned taddr = tmem + ((unsigned)(32 * warp) << 16);
#pragma unroll
        for (int c = 0; c < KD_BN / 16; ++c) {
            float v[16];
            tmem_ld16(taddr + 16 * c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j)
                g.Dp[((size_t)blockIdx.y * KD_BN + 16 * c + j) * g.mp + row] = v[j];   // coalesced over lanes
        }
    }
    tc_fence_before();
    __syncthreads();
    // copies still in flight (only after an expired wait) must land before the CTA exits
    if (tid == 0) {
        const int issued = s_issued;
        for (int s = 0; s < KD_STAGES && s < issued; ++s) {
            const int last = s + ((issued - 1 - s) / KD_STAGES) * KD_STAGES;   // last copy into stage s
            mbar_wait(&full[s], (unsigned)((last / KD_STAGES) & 1), g.timeout_ns);
        }
    }
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, KD_BN);
    }
}

// K = exp(-G / eps) (log2 form: 2^(-G kap)), BF16, and its transpose; zero padding.
__global__ void __launch_bounds__(256) kd_kmat_kernel(const float* __restrict__ G, int ld, int m, int mp, float kap,
                                                      __nv_bfloat16* __restrict__ K, __nv_bfloat16* __restrict__ Kt) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;   // column, row of the tile
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int i = by + r, j = bx + tx;
        const float v = (i < m && j < m) ? ex2(-G[(size_t)i * ld + j] * kap) : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        K[(size_t)i * mp + j] = h;
        tile[r][tx] = h;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) Kt[(size_t)(bx + r) * mp + by + tx] = tile[tx][r];
}

// Unit-mass histograms (FP32 [64][mp], zero padding), first scalings V = 1, U = 0.
__global__ void __launch_bounds__(256) kd_prep_kernel(const float* __restrict__ a, const float* __restrict__ b, int m,
                                                      int mp, int nrhs, float* __restrict__ alpha,
                                                      float* __restrict__ beta, float* __restrict__ U,
                                                      float* __restrict__ V, __nv_bfloat16* __restrict__ Ut,
                                                      __nv_bfloat16* __restrict__ Vt) {
    const int n = blockIdx.x;   // one block per right-hand side (64)
    __shared__ double red[2][8];
    double sa = 0.0, sb = 0.0;
    if (n < nrhs) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            sa += a[(size_t)n * m + i];
            sb += b[(size_t)n * m + i];
        }
    }
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sa;
        red[1][threadIdx.x >> 5] = sb;
    }
    __syncthreads();
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < 8; ++w) {
        ta += red[0][w];
        tb += red[1][w];
    }
    const float ia = ta > 0.0 ? (float)(1.0 / ta) : 0.f, ib = tb > 0.0 ? (float)(1.0 / tb) : 0.f;
    for (int i = threadIdx.x; i < mp; i += blockDim.x) {
        const bool in = n < nrhs && i < m;
        const size_t o = (size_t)n * mp + i;
        alpha[o] = in ? a[(size_t)n * m + i] * ia : 0.f;
        beta[o] = in ? b[(size_t)n * m + i] * ib : 0.f;
        U[o] = 0.f;
        V[o] = in ? 1.f : 0.f;
        Ut[o] = __float2bfloat16_rn(0.f);
        Vt[o] = __float2bfloat16_rn(in ? 1.f : 0.f);
    }
}

// X = H ./ D with D the sum of the product's reduction slices (0 where D = 0 or
// outside the problem); err[n] += sum_i |Xold_i D_i - H_i|,
// the L1 marginal error of the state before this half-iteration on this side.
__global__ void __launch_bounds__(256) kd_scale_kernel(const float* __restrict__ Dp, int splits,
                                                       const float* __restrict__ H, float* __restrict__ X,
                                                       __nv_bfloat16* __restrict__ Xt, int m, int mp,
                                                       float* __restrict__ err) {
    const int n = blockIdx.y;
    float e = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < mp; i += gridDim.x * blockDim.x) {
        const size_t o = (size_t)n * mp + i;
        float d = 0.f;   // the product: sum of the reduction slices
        for (int sl = 0; sl < splits; ++sl) d += Dp[(size_t)sl * KD_BN * mp + o];
        const float h = H[o];
        if (err) e += fabsf(fmaf(X[o], d, -h));
        const float x = (i < m && d > 0.f && h > 0.f) ? __fdiv_rn(h, d) : 0.f;
        X[o] = x;
        Xt[o] = __float2bfloat16_rn(x);
    }
    if (err) {
        e = warp_sum(e);
        if ((threadIdx.x & 31) == 0 && e != 0.f) atomicAdd(err + n, e);
    }
}

// z = eps ln V (FP64 out, [nrhs][m]); zero scalings map to the most negative finite log.
__global__ void __launch_bounds__(256) kd_log_kernel(const float* __restrict__ V, int m, int mp, int nrhs, double eps,
                                                     double* __restrict__ z) {
    const int n = blockIdx.y;
    if (n >= nrhs) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const float v = V[(size_t)n * mp + i];
        z[(size_t)n * m + i] = eps * log((double)fmaxf(v, 1e-37f));
    }
}

// ---- host side

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct KdLayout {
    size_t K, Kt, alpha, beta, U, V, Ut, Vt, D, err, flag, total;
};

static KdLayout kd_layout(int mp) {
    KdLayout L;
    size_t o = 0;
    const size_t mm = (size_t)mp * mp, vn = (size_t)KD_BN * mp;
    L.K = o; o = a256(o + 2 * mm);
    L.Kt = o; o = a256(o + 2 * mm);
    L.alpha = o; o = a256(o + 4 * vn);
    L.beta = o; o = a256(o + 4 * vn);
    L.U = o; o = a256(o + 4 * vn);
    L.V = o; o = a256(o + 4 * vn);
    L.Ut = o; o = a256(o + 2 * vn);
    L.Vt = o; o = a256(o + 2 * vn);
    L.D = o; o = a256(o + 4 * vn * KD_MAX_SPLITS);
    L.err = o; o = a256(o + 4 * (size_t)KD_BN);
    L.flag = o; o = a256(o + 64);
    L.total = o;
    return L;
}

static int kd_pad(int m) { return (m + KD_BM - 1) / KD_BM * KD_BM; }

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2-D BF16 tensor map: `rows` x `cols` row-major (row stride cols * 2 bytes), box 64 columns x box_rows rows.
static bool make_map(CUtensorMap* map, void* base, int rows, int cols, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {KD_BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Reduction slices of the product for size mp (the grid fills two resident CTAs per SM in one wave).
static int kd_splits(int mp) {
    const int sms = device_sms();
    if (sms <= 0) return 0;
    const int tiles = mp / KD_BM, nkb = mp / KD_BK;
    int splits = (2 * sms) / tiles;
    splits = splits < 1 ? 1 : (splits > nkb ? nkb : splits);
    splits = splits > KD_MAX_SPLITS ? KD_MAX_SPLITS : splits;
    const int per = (nkb + splits - 1) / splits;
    return (nkb + per - 1) / per;   // every slice non-empty
}

// Partial products Dp[s] (s < kd_splits(mp)) of A X^T for the [mp][mp] BF16 matrix behind mapA.
static int kd_gemm(const CUtensorMap& mapA, const CUtensorMap& mapX, int mp, float* Dp, int* flag,
                   unsigned long long timeout_ns, cudaStream_t st) {
    const int splits = kd_splits(mp);
    if (splits <= 0) return OT_ERR_CUDA;
    const int tiles = mp / KD_BM, nkb = mp / KD_BK;
    GemmArgs g;
    g.mp = mp;
    g.kb_per_split = (nkb + splits - 1) / splits;
    g.Dp = Dp;
    g.err = flag;
    g.timeout_ns = timeout_ns;
    kd_gemm_kernel<<<dim3(tiles, splits), 128, KD_SMEM, st>>>(mapA, mapX, g);
    return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}

}  // namespace cyc

using namespace cyc;

extern "C" size_t ot_kdomain_workspace_bytes(int m) {
    if (m <= 0 || m > 16384) return 0;
    return kd_layout(kd_pad(m)).total;
}

extern "C" int ot_kdomain_solve(int m, const float* G, int ld, float eps, int nrhs, const float* a_hist,
                                const float* b_hist, int iters, double* z_out, float* row_err, void* workspace,
                                size_t ws_bytes, void* stream) {
    if (m <= 0 || m > 16384 || !G || ld < m || !(eps > 0.f) || nrhs < 1 || nrhs > KD_BN || !a_hist || !b_hist ||
        iters < 1 || !z_out || !workspace)
        return OT_ERR_ARG;
    const int mp = kd_pad(m);
    const KdLayout L = kd_layout(mp);
    if (ws_bytes < L.total || ((uintptr_t)workspace) % 256) return OT_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)workspace;
    __nv_bfloat16* K = (__nv_bfloat16*)(w + L.K);
    __nv_bfloat16* Kt = (__nv_bfloat16*)(w + L.Kt);
    float* alpha = (float*)(w + L.alpha);
    float* beta = (float*)(w + L.beta);
    float* U = (float*)(w + L.U);
    float* V = (float*)(w + L.V);
    __nv_bfloat16* Ut = (__nv_bfloat16*)(w + L.Ut);
    __nv_bfloat16* Vt = (__nv_bfloat16*)(w + L.Vt);
    float* D = (float*)(w + L.D);
    int* flag = (int*)(w + L.flag);
    CUtensorMap mK, mKt, mU, mV;
    if (!make_map(&mK, K, mp, mp, KD_BM) || !make_map(&mKt, Kt, mp, mp, KD_BM) || !make_map(&mU, Ut, KD_BN, mp, KD_BN) ||
        !make_map(&mV, Vt, KD_BN, mp, KD_BN))
        return OT_ERR_CUDA;
    if (cudaFuncSetAttribute(kd_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, KD_SMEM) != cudaSuccess)
        return OT_ERR_CUDA;
    if (cudaMemsetAsync(flag, 0, 64, st) != cudaSuccess) return OT_ERR_CUDA;
    if (row_err && cudaMemsetAsync(row_err, 0, sizeof(float) * KD_BN * (size_t)iters, st) != cudaSuccess)
        return OT_ERR_CUDA;
    const float kap = (float)(1.0 / ((double)eps * OT_LN2));
    kd_kmat_kernel<<<dim3(mp / 32, mp / 32), 256, 0, st>>>(G, ld, m, mp, kap, K, Kt);
    kd_prep_kernel<<<KD_BN, 256, 0, st>>>(a_hist, b_hist, m, mp, nrhs, alpha, beta, U, V, Ut, Vt);
    if (cudaGetLastError() != cudaSuccess) return OT_ERR_CUDA;
    const unsigned long long tmo = 10000000000ull;
    const dim3 sgrid((mp + 255) / 256 < 64 ? (mp + 255) / 256 : 64, KD_BN);
    const int splits = kd_splits(mp);
    for (int it = 0; it < iters; ++it) {
        int rc = kd_gemm(mK, mV, mp, D, flag, tmo, st);   // D = K V (in reduction slices)
        if (rc != OT_OK) return rc;
        kd_scale_kernel<<<sgrid, 256, 0, st>>>(D, splits, alpha, U, Ut, m, mp,
                                               row_err ? row_err + (size_t)it * KD_BN : nullptr);
        rc = kd_gemm(mKt, mU, mp, D, flag, tmo, st);       // D = K^T U
        if (rc != OT_OK) return rc;
        kd_scale_kernel<<<sgrid, 256, 0, st>>>(D, splits, beta, V, Vt, m, mp, nullptr);
    }
    kd_log_kernel<<<dim3(sgrid.x, KD_BN), 256, 0, st>>>(V, m, mp, nrhs, (double)eps, z_out);
    return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}

// Reads back the error flag of the last ot_kdomain_solve on this workspace (host int).
extern "C" int ot_kdomain_status(const void* workspace, int m, int* status, void* stream) {
    if (!workspace || !status || m <= 0 || m > 16384) return OT_ERR_ARG;
    const KdLayout L = kd_layout(kd_pad(m));
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(status, (const char*)workspace + L.flag, sizeof(int), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return OT_ERR_CUDA;
    return OT_OK;
}

namespace {
__device__ int g_kd_product_flag;

__global__ void __launch_bounds__(256) kd_sum_slices_kernel(const float* __restrict__ Dp, int splits, int mp,
                                                            float* __restrict__ Dt) {
    const int n = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < mp; i += gridDim.x * blockDim.x) {
        float d = 0.f;
        for (int s = 0; s < splits; ++s) d += Dp[((size_t)s * KD_BN + n) * mp + i];
        Dt[(size_t)n * mp + i] = d;
    }
}
}

// Dt[n][i] = sum_k A[i][k] X[n][k] on the tensor cores (the product inside ot_kdomain_solve).
extern "C" int ot_kdomain_product(int mp, const void* A, const void* X, float* Dt, void* workspace, size_t ws_bytes,
                                  void* stream) {
    if (mp <= 0 || mp % KD_BM != 0 || mp > 16384 || !A || !X || !Dt || !workspace) return OT_ERR_ARG;
    if (((uintptr_t)A) % 16 || ((uintptr_t)X) % 16) return OT_ERR_ARG;
    const KdLayout L = kd_layout(mp);
    if (ws_bytes < L.total || ((uintptr_t)workspace) % 256) return OT_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    CUtensorMap mA, mX;
    if (!make_map(&mA, (void*)A, mp, mp, KD_BM) || !make_map(&mX, (void*)X, KD_BN, mp, KD_BN)) return OT_ERR_CUDA;
    if (cudaFuncSetAttribute(kd_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, KD_SMEM) != cudaSuccess)
        return OT_ERR_CUDA;
    int* flag = nullptr;
    if (cudaGetSymbolAddress((void**)&flag, g_kd_product_flag) != cudaSuccess) return OT_ERR_CUDA;
    if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return OT_ERR_CUDA;
    // the slices go to the workspace's product region, then one pass sums them into Dt
    const int splits = kd_splits(mp);
    if (splits <= 0) return OT_ERR_CUDA;
    float* Dp = (float*)((char*)workspace + L.D);
    int rc = kd_gemm(mA, mX, mp, Dp, flag, 10000000000ull, st);
    if (rc != OT_OK) return rc;
    kd_sum_slices_kernel<<<dim3((mp + 255) / 256 < 64 ? (mp + 255) / 256 : 64, KD_BN), 256, 0, st>>>(Dp, splits, mp, Dt);
    if (cudaGetLastError() != cudaSuccess) return OT_ERR_CUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return OT_ERR_CUDA;
    return h;
}
