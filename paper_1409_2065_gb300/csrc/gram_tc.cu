// Gram matrix G = Y Y^T on the tensor cores (placeholder until the tcgen05
// kernel lands): reports "not supported" so the caller uses the FP32 kernel.
#include <cuda_runtime.h>

namespace ccx {

cudaError_t launch_gram_tc(const float* Y, int n, int p, int ld, float* G, double* unit, cudaStream_t s) {
    (void)Y; (void)n; (void)p; (void)ld; (void)G; (void)unit; (void)s;
    return cudaErrorNotSupported;
}

}  // namespace ccx
