// Unrolled-iteration adjoint (placeholder until the reverse-pass kernel lands).
#include "common.cuh"

namespace cyc {

size_t unrolled_ws_bytes(int m, int N, int iters) { return 256; }

int run_unrolled(int, int, const float*, const float*, const float*, const float*, const float*, const float*, float,
                 int, ot_result*, float*, float*, float*, float*, float*, void*, size_t, cudaStream_t) {
    return OT_ERR_UNSUPPORTED;
}

}  // namespace cyc
