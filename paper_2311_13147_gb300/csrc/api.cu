// Library-wide entry points: version, status names, workspace sizes, device queries.
#include "common.cuh"

namespace cyc {

size_t solver_ws_bytes(int M, int Ncol, bool stored);
size_t value_ws_bytes(int m);
size_t unrolled_ws_bytes(int m, int N, int iters);

// SM count of the current device, cached per device.
int device_sms() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
    if (dev < 64 && cache[dev] > 0) return cache[dev];
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (dev < 64) cache[dev] = sms;
    return sms;
}

}  // namespace cyc

using namespace cyc;

extern "C" const char* ot_version(void) { return "cyclicot 0.1 sm_103a"; }

extern "C" const char* ot_status_string(int s) {
    switch (s) {
        case OT_OK: return "OT_OK";
        case OT_ERR_ARG: return "OT_ERR_ARG: invalid argument";
        case OT_ERR_NOT_DIVISIBLE: return "OT_ERR_NOT_DIVISIBLE: n is not a multiple of N";
        case OT_ERR_NOT_CONVERGED: return "OT_ERR_NOT_CONVERGED: max_iter reached";
        case OT_ERR_TIMEOUT: return "OT_ERR_TIMEOUT: a device-side wait expired";
        case OT_ERR_NONFINITE: return "OT_ERR_NONFINITE: NaN or Inf in the iteration";
        case OT_ERR_CUDA: return "OT_ERR_CUDA: CUDA runtime error";
        case OT_ERR_WORKSPACE: return "OT_ERR_WORKSPACE: workspace missing, misaligned or too small";
        case OT_ERR_UNSUPPORTED: return "OT_ERR_UNSUPPORTED: size or mode not supported";
        default: return "unknown status";
    }
}

extern "C" size_t ot_workspace_bytes(int op, int m_or_n, int N, const ot_options* opt) {
    if (m_or_n <= 0 || N <= 0) return 0;
    switch (op) {
        case OT_OP_SINKHORN_REDUCED: return solver_ws_bytes(m_or_n, m_or_n, true);
        case OT_OP_SINKHORN_FULL: return solver_ws_bytes(m_or_n, m_or_n, true);
        case OT_OP_VALUE_AND_GRAD: return value_ws_bytes(m_or_n);
        case OT_OP_UNROLLED: return unrolled_ws_bytes(m_or_n, N, opt ? opt->max_iter : 200);
        default: return 0;
    }
}
