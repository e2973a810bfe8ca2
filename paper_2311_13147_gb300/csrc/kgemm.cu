// Kernel-domain Sinkhorn on 64 right-hand sides sharing one folded cost, with
// the two matrix products of every iteration on the tcgen05 tensor cores.
//
// Algorithm 2 written in scaling form (the closed forms of Eq.
// optimal_f_sinkhorn_logdomain exponentiated): with K = exp(-G^eps / eps) and
// marginals alpha_n, beta_n of unit mass, one iteration is
//     U = alpha ./ (K V),    V = beta ./ (K^T U)
// for all 64 histogram pairs n at once, i.e. two [m x m] x [m x 64] products.
// K and K^T are stored as BF16 (padded to mp, a multiple of 128) in tile-major
// order, so that each pipeline stage's [128 x 64] tile is 16 KB of contiguous
// memory (one DRAM stream per stage instead of 128 rows of 128 bytes); the products
// accumulate in FP32 in tensor memory.  BF16 limits the fixed point's accuracy
// to about 1e-3; the FP32 log-domain batch solver then polishes each pair from
// z = eps log V (warm start) to the requested tolerance.
//
// GEMM kernel (one 128-row tile of the output and one slice of the reduction
// per CTA, 128 threads; the slices of a tile form one thread-block cluster):
//   thread 0      TMA producer: K tile [128 x 64] and scaling tile [64 x 64]
//                 per 64-wide reduction block into a 4-stage ring (128-byte
//                 swizzle), completion counted on the stage's mbarrier;
//   thread 32     MMA issuer: 4 tcgen05.mma (M 128, N 64, K 16, BF16 -> FP32)
//                 per stage, then tcgen05.commit frees the stage;
//   all 4 warps   epilogue: tcgen05.ld of the 128 x 64 FP32 accumulator (warp w
//                 reads lanes 32w..32w+31) into this CTA's shared memory (the
//                 free pipeline stages); after a cluster barrier, CTA r of the
//                 cluster sums the slices of its share of the 64 right-hand
//                 sides from its peers' shared memory (distributed shared
//                 memory, slices in order) and writes either the product or,
//                 in the solver, the scaling update X = H ./ D of those columns;
//                 a second cluster barrier keeps every slice readable until
//                 its peers are done.  No partial product touches global memory.
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
#define KD_MAX_SPLITS 8            // reduction slices = cluster size (portable limit), a power of two

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

// Cluster barrier (every thread of every CTA of the cluster arrives); release and
// acquire order the shared-memory writes before it with the peer reads after it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// The address of the same shared-memory location in CTA `rank` of this cluster.
__device__ __forceinline__ unsigned dsmem_addr(unsigned local, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}

// (volatile: stays after the cluster barrier; no memory clobber, so the loads of a
// chunk can all be in flight together)
__device__ __forceinline__ float ld_dsmem(unsigned addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

// Programmatic dependent launch: wait until the preceding grid of the stream has
// completed and its writes are visible (returns at once without a preceding
// dependent-launch edge); allow the next grid to begin launching.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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
    int a_tiled;                  // A in tile-major order (kd_tiled) rather than row-major
    int* err;                     // error flag (OT_ERR_TIMEOUT on an expired wait)
    unsigned long long timeout_ns;
    float* D;                     // [64][mp] product output (H == nullptr)
    // scaling update (H != nullptr): X = H ./ D, 0 where D = 0, H = 0 or i >= m
    const float* H;               // [64][mp] target histograms (alpha or beta)
    float* X;                     // [64][mp] scaling, updated in place (U or V)
    __nv_bfloat16* Xt;            // [64][mp] its BF16 copy, the next product's operand
    float* row_err;               // [64] += sum_i |Xold_i D_i - H_i| (the state before the update), or nullptr
    int m;                        // problem size (rows >= m are padding)
};

// D[n][i] = sum_k A[i][k] X[n][k] for this cluster's 128 rows i, reduced over the
// cluster's slices of k, then written or turned into the scaling update.
// A: tensor map of a [mp][mp] BF16 matrix (row-major, K-major operand);
// X: tensor map of the [64][mp] BF16 scaling vectors (K-major operand).
// Grid (mp / 128, splits), cluster (1, splits, 1); slice y covers reduction
// blocks [y nkb / splits, (y + 1) nkb / splits), never empty (splits <= nkb).
template <int SPLITS>
__global__ void __launch_bounds__(128, 1) kd_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmX, GemmArgs g) {
    extern __shared__ unsigned char kd_smem_raw[];
    __shared__ __align__(8) unsigned long long full[KD_STAGES], empty[KD_STAGES], accb;
    __shared__ unsigned tmem_slot;
    __shared__ int s_issued;
    __shared__ float s_err[KD_BN];
    unsigned char* base =
        (unsigned char*)(((uintptr_t)kd_smem_raw + 1023) & ~(uintptr_t)1023);   // 1024-byte aligned tiles
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * KD_BM;
    const int nkb_total = g.mp / KD_BK, splits = SPLITS;
    const int kb0 = (int)((blockIdx.y * nkb_total) / splits);
    const int kb1 = (int)(((blockIdx.y + 1) * nkb_total) / splits);
    const int nkb = kb1 - kb0;   // >= 1 (the host keeps splits <= nkb_total)

    if (tid == 0) {
        for (int s = 0; s < KD_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accb, 1);
        fence_mbar_init();
    }
    if (tid < KD_BN) s_err[tid] = 0.f;
    if (warp == 1) tmem_alloc(&tmem_slot, KD_BN);   // 64 FP32 columns x 128 lanes
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;

    // a launch queued behind this one (programmatic dependent launch) may start its own
    // prologue now; it reads nothing this grid writes before its griddepcontrol.wait
    grid_dep_launch();

    if (warp == 0 && lane == 0) {
        // producer.  The matrix tiles of the first stages depend on no earlier launch of
        // the solve (K and K^T are written once, before the first product, which is
        // launched without the dependent-launch attribute): they are requested before
        // waiting for the previous product, whose scaling update the X tiles read.
        const int pre = min(nkb, KD_STAGES);
        // the A tile of reduction block kb: tile-major (one 16 KB run) or row-major
        const int a_col = g.a_tiled ? 0 : -1;
        const int a_row0 = g.a_tiled ? (int)blockIdx.x * nkb_total * KD_BM : m0;
        for (int i = 0; i < pre; ++i) {
            const int kb = kb0 + i;
            mbar_arrive_expect_tx(&full[i], KD_STAGE_BYTES);
            tma_load_2d(base + (size_t)i * KD_STAGE_BYTES, &tmA, a_col < 0 ? kb * KD_BK : 0,
                        a_col < 0 ? a_row0 : a_row0 + kb * KD_BM, &full[i]);
        }
        grid_dep_wait();
        for (int i = 0; i < pre; ++i)
            tma_load_2d(base + (size_t)i * KD_STAGE_BYTES + KD_A_BYTES, &tmX, (kb0 + i) * KD_BK, 0, &full[i]);
        int i = pre;
        for (; i < nkb; ++i) {
            const int s = i % KD_STAGES;
            const unsigned ph = (unsigned)((i / KD_STAGES) & 1);
            if (!mbar_wait(&empty[s], ph ^ 1u, g.timeout_ns)) {
                atomicExch(g.err, OT_ERR_TIMEOUT);
                break;
            }
            unsigned char* st = base + (size_t)s * KD_STAGE_BYTES;
            mbar_arrive_expect_tx(&full[s], KD_STAGE_BYTES);
            const int kb = kb0 + i, kc = kb * KD_BK;
            tma_load_2d(st, &tmA, a_col < 0 ? kc : 0, a_col < 0 ? a_row0 : a_row0 + kb * KD_BM, &full[s]);
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
    grid_dep_wait();   // the previous launch's writes are visible before H, X and D are touched
    // this CTA's share of the right-hand sides, n in [n0, n0 + NPER), in chunks of CH
    constexpr int NPER = KD_BN / SPLITS, CH = NPER < 32 ? NPER : 32;
    const int n0 = (int)blockIdx.y * NPER;   // blockIdx.y is the rank in the cluster
    const int i = m0 + tid;
    float h[CH], xo[CH];   // the first chunk's histogram and old scaling, fetched while the MMAs run
    if (g.H) {
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const size_t o = (size_t)(n0 + j) * g.mp + i;
            h[j] = g.H[o];
            xo[j] = g.row_err ? g.X[o] : 0.f;
        }
    }
    const bool ok = mbar_wait(&accb, 0u, g.timeout_ns);
    if (!ok && lane == 0) atomicExch(g.err, OT_ERR_TIMEOUT);
    tc_fence_after();
    // copies still in flight (only after an expired wait) land before the stages are reused
    if (tid == 0) {
        const int issued = s_issued;
        for (int s = 0; s < KD_STAGES && s < issued; ++s) {
            const int last = s + ((issued - 1 - s) / KD_STAGES) * KD_STAGES;   // last copy into stage s
            mbar_wait(&full[s], (unsigned)((last / KD_STAGES) & 1), g.timeout_ns);
        }
    }
    __syncthreads();   // every MMA has read its stage (accb) and every copy has landed
    // this slice's partial product, [64][128] FP32 in the first 32 KB of the stages
    float* part = reinterpret_cast<float*>(base);
    {
        const bool all_ok = __all_sync(0xffffffffu, ok);
        const unsigned taddr = tmem + ((unsigned)(32 * warp) << 16);
#pragma unroll
        for (int c = 0; c < KD_BN / 16; ++c) {
            float v[16];
            if (all_ok) {
                tmem_ld16(taddr + 16 * c, v);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0.f;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) part[(16 * c + j) * KD_BM + tid] = v[j];   // conflict-free over lanes
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, KD_BN);
    }
    cluster_sync();   // every slice of the tile is in its CTA's shared memory

    const unsigned part_local = smem_addr(part + tid);
#pragma unroll 1
    for (int nc = 0; nc < NPER; nc += CH) {
        if (nc > 0 && g.H) {
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const size_t o = (size_t)(n0 + nc + j) * g.mp + i;
                h[j] = g.H[o];
                xo[j] = g.row_err ? g.X[o] : 0.f;
            }
        }
        // every slice's values first (all loads in flight), then the sums in slice order
        float v[SPLITS][CH];
#pragma unroll
        for (int sl = 0; sl < SPLITS; ++sl) {
            const unsigned pa = dsmem_addr(part_local, (unsigned)sl) + (unsigned)((n0 + nc) * KD_BM * 4);
#pragma unroll
            for (int j = 0; j < CH; ++j) v[sl][j] = ld_dsmem(pa + (unsigned)(j * KD_BM * 4));
        }
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            float d = 0.f;
#pragma unroll
            for (int sl = 0; sl < SPLITS; ++sl) d += v[sl][j];
            const int n = n0 + nc + j;
            const size_t o = (size_t)n * g.mp + i;
            if (!g.H) {
                g.D[o] = d;
                continue;
            }
            const float x = (i < g.m && d > 0.f && h[j] > 0.f) ? __fdiv_rn(h[j], d) : 0.f;
            if (g.row_err) {
                const float e = warp_sum(fabsf(fmaf(xo[j], d, -h[j])));
                if (lane == 0 && e != 0.f) atomicAdd(&s_err[n], e);
            }
            g.X[o] = x;
            g.Xt[o] = __float2bfloat16_rn(x);
        }
    }
    if (g.row_err) {
        __syncthreads();
        if (tid < NPER && s_err[n0 + tid] != 0.f) atomicAdd(g.row_err + n0 + tid, s_err[n0 + tid]);
    }
    cluster_sync();   // the peers have read this CTA's slice
}

// Tile-major offset of element (i, j) of an [mp][mp] operand: [128 x 64] tiles,
// those of a row block consecutive, rows of 64 within a tile.
__device__ __forceinline__ size_t kd_tiled(int i, int j, int mp) {
    return ((size_t)(i >> 7) * (size_t)(mp >> 6) + (size_t)(j >> 6)) * (KD_BM * KD_BK) + (size_t)((i & 127) * KD_BK + (j & 63));
}

// K = exp(-G / eps) (log2 form: 2^(-G kap)), BF16, and its transpose, both tile-major; zero padding.
__global__ void __launch_bounds__(256) kd_kmat_kernel(const float* __restrict__ G, int ld, int m, int mp, float kap,
                                                      __nv_bfloat16* __restrict__ K, __nv_bfloat16* __restrict__ Kt) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;   // column, row of the tile
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int i = by + r, j = bx + tx;
        const float v = (i < m && j < m) ? ex2(-G[(size_t)i * ld + j] * kap) : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        K[kd_tiled(i, j, mp)] = h;
        tile[r][tx] = h;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) Kt[kd_tiled(bx + r, by + tx, mp)] = tile[tx][r];
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
    size_t K, Kt, alpha, beta, U, V, Ut, Vt, err, flag, total;
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

// Reduction slices of the product for size mp: the largest power of two <= 8 that keeps
// the grid within two resident CTAs per SM (one wave) and every slice non-empty.
static int kd_splits(int mp) {
    const int sms = device_sms();
    if (sms <= 0) return 0;
    const int tiles = mp / KD_BM, nkb = mp / KD_BK;
    int splits = 1;
    while (splits * 2 <= KD_MAX_SPLITS && splits * 2 <= nkb && tiles * splits * 2 <= 2 * sms) splits *= 2;
    return splits;
}

// One product of the [mp][mp] BF16 matrix behind mapA with the scalings behind mapX:
// g.H == nullptr writes D = A X^T to g.D, else the scaling update (g's other fields).
// pdl: launch as a programmatic dependent of the previous kernel in the stream, which must
// not write mapA's matrix (the previous product of the solve).
static int kd_gemm(const CUtensorMap& mapA, const CUtensorMap& mapX, int mp, GemmArgs g, int* flag,
                   unsigned long long timeout_ns, cudaStream_t st, bool pdl = false) {
    const int splits = kd_splits(mp);
    if (splits <= 0) return OT_ERR_CUDA;
    g.mp = mp;
    g.err = flag;
    g.timeout_ns = timeout_ns;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(mp / KD_BM, splits, 1);
    cfg.blockDim = dim3(128, 1, 1);
    cfg.dynamicSmemBytes = KD_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = (unsigned)splits;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    cudaError_t e;
    switch (splits) {
        case 1: e = cudaLaunchKernelEx(&cfg, kd_gemm_kernel<1>, mapA, mapX, g); break;
        case 2: e = cudaLaunchKernelEx(&cfg, kd_gemm_kernel<2>, mapA, mapX, g); break;
        case 4: e = cudaLaunchKernelEx(&cfg, kd_gemm_kernel<4>, mapA, mapX, g); break;
        case 8: e = cudaLaunchKernelEx(&cfg, kd_gemm_kernel<8>, mapA, mapX, g); break;
        default: return OT_ERR_CUDA;
    }
    return e == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}

// The GEMM kernels' shared-memory opt-in.
static bool kd_gemm_attrs() {
    return cudaFuncSetAttribute(kd_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, KD_SMEM) ==
               cudaSuccess &&
           cudaFuncSetAttribute(kd_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, KD_SMEM) ==
               cudaSuccess &&
           cudaFuncSetAttribute(kd_gemm_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, KD_SMEM) ==
               cudaSuccess &&
           cudaFuncSetAttribute(kd_gemm_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, KD_SMEM) ==
               cudaSuccess;
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
    int* flag = (int*)(w + L.flag);
    CUtensorMap mK, mKt, mU, mV;
    // K and K^T tile-major: a [mp mp / 64][64] view whose [128 x 64] boxes are whole tiles
    const int trows = (int)((size_t)mp * mp / KD_BK);
    if (!make_map(&mK, K, trows, KD_BK, KD_BM) || !make_map(&mKt, Kt, trows, KD_BK, KD_BM) ||
        !make_map(&mU, Ut, KD_BN, mp, KD_BN) ||
        !make_map(&mV, Vt, KD_BN, mp, KD_BN))
        return OT_ERR_CUDA;
    if (!kd_gemm_attrs()) return OT_ERR_CUDA;
    if (cudaMemsetAsync(flag, 0, 64, st) != cudaSuccess) return OT_ERR_CUDA;
    if (row_err && cudaMemsetAsync(row_err, 0, sizeof(float) * KD_BN * (size_t)iters, st) != cudaSuccess)
        return OT_ERR_CUDA;
    const float kap = (float)(1.0 / ((double)eps * OT_LN2));
    kd_kmat_kernel<<<dim3(mp / 32, mp / 32), 256, 0, st>>>(G, ld, m, mp, kap, K, Kt);
    kd_prep_kernel<<<KD_BN, 256, 0, st>>>(a_hist, b_hist, m, mp, nrhs, alpha, beta, U, V, Ut, Vt);
    if (cudaGetLastError() != cudaSuccess) return OT_ERR_CUDA;
    const unsigned long long tmo = 10000000000ull;
    const dim3 sgrid((mp + 255) / 256 < 64 ? (mp + 255) / 256 : 64, KD_BN);
    GemmArgs gu = {}, gv = {};
    gu.a_tiled = gv.a_tiled = 1;
    gu.m = gv.m = m;
    gu.H = alpha, gu.X = U, gu.Xt = Ut;   // U = alpha ./ (K V)
    gv.H = beta, gv.X = V, gv.Xt = Vt;    // V = beta ./ (K^T U)
    for (int it = 0; it < iters; ++it) {
        gu.row_err = row_err ? row_err + (size_t)it * KD_BN : nullptr;
        int rc = kd_gemm(mK, mV, mp, gu, flag, tmo, st, it > 0);
        if (rc != OT_OK) return rc;
        rc = kd_gemm(mKt, mU, mp, gv, flag, tmo, st, true);
        if (rc != OT_OK) return rc;
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
    if (!kd_gemm_attrs()) return OT_ERR_CUDA;
    int* flag = nullptr;
    if (cudaGetSymbolAddress((void**)&flag, g_kd_product_flag) != cudaSuccess) return OT_ERR_CUDA;
    if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return OT_ERR_CUDA;
    GemmArgs g = {};
    g.D = Dt;
    int rc = kd_gemm(mA, mX, mp, g, flag, 10000000000ull, st);
    if (rc != OT_OK) return rc;
    int h = 0;
    if (cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return OT_ERR_CUDA;
    return h;
}
