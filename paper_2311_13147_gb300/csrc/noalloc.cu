// ot_sinkhorn_reduced_static: the reduced-problem solver with a scratch area
// that the library owns, for callers that cannot allocate device memory.
//
// Some callers have no way to obtain device memory at the point of the call:
// a plugin running inside a host framework that owns the device allocator and
// forbids direct cudaMalloc, or a latency-bound loop that must not allocate
// after start-up (cudaMalloc can synchronise the device and takes unbounded
// time).  Such callers still pass their inputs and outputs; the scratch space
// that ot_sinkhorn_reduced takes as `workspace` comes instead from a fixed
// array compiled into this library.
//
// Limits and sharing:
// - The array holds kStaticScratchBytes (4 MiB).  Each call compares that with
//   ot_workspace_bytes for its (m, N, options), which grows with m and with the
//   device's SM count; requests that do not fit are rejected with
//   OT_ERR_UNSUPPORTED before anything is launched.  On a 152-SM GB300 every
//   m <= 4096 fits.
// - Every GPU that loads the library holds its own copy of the array until
//   the process exits.
// - All calls on a device share that one array and it keeps the contents of
//   the last call.  The solver clears what must start at zero (its control
//   block and its accumulation vectors) at the start of every call, so
//   consecutive calls are independent; calls that overlap on the GPU (for
//   example on two streams at once) race on the array and give wrong results.
// - The first call on a device looks up the array's device address with
//   cudaGetSymbolAddress (that device must be current); make that first call
//   before any stream capture begins.  The address is kept for the rest of the
//   process, so resetting the device (cudaDeviceReset) after that first call is
//   not supported: the module is loaded again and the array may move.
// - Neither this entry point nor anything it calls allocates memory.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kStaticScratchBytes = 4u << 20;

// One copy per device; in host code this name is only a host-side stand-in,
// the device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[64] = {};

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return OT_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return OT_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return OT_OK;
}

}  // namespace

extern "C" int ot_sinkhorn_reduced_static(int m, int N, const float* a_base, const float* b_base, const float* G,
                                          const ot_options* opt, double* w, double* z, ot_result* out,
                                          void* stream) {
    if (m <= 0 || N <= 0 || opt == nullptr) return OT_ERR_ARG;
    const size_t need = ot_workspace_bytes(OT_OP_SINKHORN_REDUCED, m, N, opt);
    if (need == 0) return OT_ERR_CUDA;
    if (need > kStaticScratchBytes) return OT_ERR_UNSUPPORTED;
    void* scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != OT_OK) return rc;
    return ot_sinkhorn_reduced(m, N, a_base, b_base, G, opt, w, z, out, scratch, kStaticScratchBytes, stream);
}
