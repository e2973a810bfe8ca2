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

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_int(const int* p) {
    return *((const volatile int*)p);
}

// Control block at the start of every persistent-kernel workspace.  The host
// zeroes it (cudaMemsetAsync) before each launch.
struct Ctrl {
    unsigned count;      // arrivals at the current barrier
    unsigned gen;        // barrier generation
    int status;          // first device-side error (OT_ERR_*), 0 if none
    int flag;            // kernel-specific shared flag
    unsigned long long pad[6];
};
static_assert(sizeof(Ctrl) == 64, "Ctrl must stay 64 bytes");

// Grid-wide barrier for a cooperative launch.  Returns false (in every thread
// of the block) if the wait expired or another block already recorded an
// error; the caller must then leave the kernel.
__device__ __forceinline__ bool grid_sync(Ctrl* c, unsigned nblocks, unsigned long long timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        unsigned g = ld_acquire(&c->gen);
        unsigned old = atomicAdd(&c->count, 1u);
        if (old == nblocks - 1) {
            c->count = 0;
            __threadfence();
            st_release(&c->gen, g + 1);
        } else {
            unsigned long long t0 = globaltimer();
            while (ld_acquire(&c->gen) == g) {
                if (globaltimer() - t0 > timeout_ns) {
                    atomicCAS(&c->status, 0, OT_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
        __threadfence();
        if (ld_volatile_int(&c->status) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void set_status(Ctrl* c, int st) { atomicCAS(&c->status, 0, st); }

// Fault injection for tests: instead of arriving at the barrier, wait (bounded)
// until another block has recorded an error, then report failure.
__device__ __forceinline__ bool withhold_arrival(Ctrl* c, unsigned long long timeout_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer();
        while (ld_volatile_int(&c->status) == 0) {
            if (globaltimer() - t0 > 4 * timeout_ns + 1000000ull) {
                atomicCAS(&c->status, 0, OT_ERR_TIMEOUT);
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
