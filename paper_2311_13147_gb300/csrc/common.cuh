// Device helpers shared by the cyclicot kernels (sm_103a).
//
// - log2-domain arithmetic on the MUFU unit: ex2.approx / lg2.approx PTX
//   instructions (hardware instructions, no library math code);
// - a grid-wide barrier for persistent cooperative kernels whose wait is
//   bounded by %globaltimer: on expiry it records OT_ERR_TIMEOUT in the
//   control block and returns false, so no kernel can hang;
// - warp / block reductions with a fixed order (deterministic results).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cyclicot.h"

#define OT_LN2 0.69314718055994530942
#define OT_BLOCK 256
#define OT_WARPS (OT_BLOCK / 32)

namespace cyc {

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_int(const int* p) {
    return *((const volatile int*)p);
}

// Control block at the start of every persistent-kernel workspace.  The host
// zeroes it (cudaMemsetAsync) before each launch.
struct Ctrl {
    unsigned count;      // monotonic barrier arrival counter (low half of the barrier word)
    unsigned gen;        // error marks (high half of the barrier word: nonzero once an error is recorded)
    int status;          // first device-side error (OT_ERR_*), 0 if none
    int flag;            // kernel-specific shared flag
    unsigned long long pad[6];
};
static_assert(sizeof(Ctrl) == 64, "Ctrl must stay 64 bytes");

// The barrier word: count (arrivals) and gen (error marks) as one 64-bit location, so a
// single acquire load tells a waiting block both whether the barrier completed and
// whether an error was recorded.
__device__ __forceinline__ unsigned long long* ctrl_word(Ctrl* c) {
    return reinterpret_cast<unsigned long long*>(&c->count);
}
__device__ __forceinline__ void red_release_add64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Records the first device-side error (its code in status) and marks the barrier word,
// so that every block waiting at a grid barrier, now or later, leaves at once.
__device__ __forceinline__ void set_status(Ctrl* c, int st) {
    atomicCAS(&c->status, 0, st);
    red_release_add64(ctrl_word(c), 1ull << 32);
}

// Grid-wide barrier for a cooperative launch.  `epoch` counts the barriers this
// block has passed (start at 0, the caller keeps it): arrivals accumulate on a
// monotonic counter and barrier k completes when it reaches nblocks * (k + 1).
// Returns false (in every thread of the block) if the wait expired or an error is
// marked (checked by the same load that observes the arrivals: no extra round trip);
// the caller must then leave the kernel.
__device__ __forceinline__ bool grid_sync(Ctrl* c, unsigned nblocks, unsigned long long timeout_ns,
                                          unsigned& epoch) {
    __shared__ int s_ok;
    __syncthreads();
    epoch += 1;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = nblocks * epoch;
        unsigned long long* wd = ctrl_word(c);
        red_release_add64(wd, 1ull);
        unsigned long long w = ld_acquire64(wd);
        if ((int)((unsigned)w - target) < 0 && (w >> 32) == 0) {
            const unsigned long long t0 = globaltimer();
            for (;;) {
                w = ld_acquire64(wd);
                if ((int)((unsigned)w - target) >= 0 || (w >> 32) != 0) break;
                if (globaltimer() - t0 > timeout_ns) {
                    set_status(c, OT_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        if ((w >> 32) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---- mbarrier + bulk async copy (TMA 1D) helpers ------------------------------

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bulk copy global -> shared, completion counted on `bar` (bytes, dst, src 16-byte multiples/aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false on expiry.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned long long timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > timeout_ns) return false;
    }
    return true;
}


// Fault injection for tests: instead of arriving at the barrier, wait (bounded)
// until another block has recorded an error, then report failure.
__device__ __forceinline__ bool withhold_arrival(Ctrl* c, unsigned long long timeout_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer();
        while (ld_volatile_int(&c->status) == 0) {
            if (globaltimer() - t0 > 4 * timeout_ns + 1000000ull) {
                set_status(c, OT_ERR_TIMEOUT);
                break;
            }
            __nanosleep(100);
        }
    }
    __syncthreads();
    return false;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Deterministic block sum of one double (all threads get the result).
__device__ __forceinline__ double block_sum_d(double v, double* red /* >= OT_WARPS */) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < OT_WARPS; ++w) t += red[w];
    return t;
}

// Split x into float hi + float lo with hi = fl(x), lo = fl(x - hi).
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

}  // namespace cyc
