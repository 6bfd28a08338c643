// Per-edge fusion ratios written into a fixed device buffer that is part of the
// library image, so that ccx_fusion_scale_noalloc needs no device allocation.
//
// The buffer is one file-scope array shared by every call on a device: a call
// overwrites entries [0, m) before it reads them, so nothing has to start at
// zero, and two calls whose kernels overlap on the GPU race on it.  Its device
// address is looked up once per device and kept; it belongs to the context that
// was current then, so it is not valid after a device reset in the process.
#include <cuda_runtime.h>

#include <mutex>

#include "ccx_internal.h"

namespace ccx {
namespace {

__device__ __align__(256) double g_edge_ratio[kStaticEdgesMax];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
double* g_addr[kMaxDevices] = {};

// One warp per edge: r_e = ||y_i - y_j|| / (2 w_e), the sum of squares in double.
__global__ void edge_ratio_kernel(const float* __restrict__ Y, int p, int ld, const int* __restrict__ ei,
                                  const int* __restrict__ ej, const double* __restrict__ w, int m,
                                  double* __restrict__ r) {
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (e >= m) return;
    const float* a = Y + (size_t)ei[e] * ld;
    const float* b = Y + (size_t)ej[e] * ld;
    double s = 0.0;
    for (int c = lane; c < p; c += 32) {
        const double dd = (double)a[c] - (double)b[c];
        s += dd * dd;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) r[e] = sqrt(s) / (2.0 * w[e]);
}

}  // namespace

cudaError_t static_edge_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_edge_ratio);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double*>(ptr);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

cudaError_t edge_ratios_static(const float* Y0f, int p, int ld, const int* ei_d, const int* ej_d, const double* w_d,
                               int m, double* scratch, cudaStream_t s) {
    if (m < 0 || m > kStaticEdgesMax) return cudaErrorInvalidValue;
    if (m == 0) return cudaSuccess;
    count_launches(1);
    edge_ratio_kernel<<<(m + 7) / 8, 256, 0, s>>>(Y0f, p, ld, ei_d, ej_d, w_d, m, scratch);
    return cudaGetLastError();
}

}  // namespace ccx
