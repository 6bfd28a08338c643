// Input packing and the start matrix Y_0.
//
// pack_input: copies the caller's X (n x p floats, stride ld_in, already on
// the device) into the internal padded layout (stride ld, padding = 0), sets
// missing entries to 0, bit-packs the mask (padding marked observed) and
// counts non-finite observed entries and rows without any observed entry.
//
// standardize: each column centred on the mean of its observed entries and
// divided by their standard deviation (divisor = their count; centred only when
// that deviation is 0), in double and rounded once (Methods: the predictors are
// standardised).
//
// fill_missing: Y_0 = X with each missing entry replaced by its column's
// observed mean (Methods, "Missing Data", start of the iteration; also the
// fill used for the weights), and ||Y_c||_F^2, the squared Frobenius norm of
// the column-centred Y_0, in double with a fixed summation order.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "ccx_internal.h"

namespace ccx {
namespace {

__global__ void pack_values_kernel(const float* __restrict__ X, const uint8_t* __restrict__ mask, int64_t n,
                                   int64_t p, int64_t ld_in, float* __restrict__ Xf, double* __restrict__ Xd, int ld,
                                   int* bad) {
    const size_t total = (size_t)n * ld;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int64_t i = (int64_t)(k / ld), c = (int64_t)(k % ld);
        float v = 0.f;
        if (c < p) {
            const bool obs = mask ? (mask[i * ld_in + c] != 0) : true;
            if (obs) {
                v = X[i * ld_in + c];
                if (!isfinite(v)) {
                    atomicAdd(bad, 1);
                    v = 0.f;
                }
            }
        }
        Xf[k] = v;
        if (Xd) Xd[k] = (double)v;
    }
}

__global__ void pack_mask_kernel(const uint8_t* __restrict__ mask, int64_t n, int64_t p, int64_t ld_in,
                                 uint32_t* __restrict__ bits, int ldw, int* empty_rows) {
    // one block per row: build the words and count observed entries
    const int64_t i = blockIdx.x;
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int local = 0;
    for (int wd = threadIdx.x; wd < ldw; wd += blockDim.x) {
        uint32_t word = 0u;
        for (int b = 0; b < 32; ++b) {
            const int64_t c = (int64_t)wd * 32 + b;
            bool obs = true;
            if (c < p) {
                obs = mask[i * ld_in + c] != 0;
                local += obs ? 1 : 0;
            }
            if (obs) word |= (1u << b);
        }
        bits[(size_t)i * ldw + wd] = word;
    }
    atomicAdd(&cnt, local);   // integer count: order does not matter
    __syncthreads();
    if (threadIdx.x == 0 && cnt == 0) atomicAdd(empty_rows, 1);
}

__global__ void column_mean_kernel(const float* __restrict__ Xf, const uint32_t* __restrict__ bits, int n, int p,
                                   int ld, int ldw, double* __restrict__ colmean) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p) return;
    double s = 0.0;
    int cnt = 0;
    for (int i = 0; i < n; ++i) {
        const bool obs = bits ? ((bits[(size_t)i * ldw + (c >> 5)] >> (c & 31)) & 1u) : true;
        if (obs) {
            s += (double)Xf[(size_t)i * ld + c];
            ++cnt;
        }
    }
    colmean[c] = cnt > 0 ? s / cnt : 0.0;
}

__global__ void fill_kernel(const float* __restrict__ Xf, const uint32_t* __restrict__ bits, int n, int p, int ld,
                            int ldw, const double* __restrict__ colmean, float* __restrict__ Y0f,
                            double* __restrict__ Y0d) {
    const size_t total = (size_t)n * ld;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k / ld), c = (int)(k % ld);
        double y = 0.0;
        if (c < p) {
            const bool obs = bits ? ((bits[(size_t)i * ldw + (c >> 5)] >> (c & 31)) & 1u) : true;
            y = obs ? (double)Xf[k] : colmean[c];
        }
        if (Y0f) Y0f[k] = (float)y;
        if (Y0d) Y0d[k] = y;
    }
}

// observed mean and standard deviation of each column (two passes in double)
__global__ void column_stats_kernel(const float* __restrict__ Xf, const uint32_t* __restrict__ bits, int n, int p,
                                    int ld, int ldw, double* __restrict__ mean, double* __restrict__ scale) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p) return;
    double s = 0.0;
    int cnt = 0;
    for (int i = 0; i < n; ++i) {
        if (bits && !((bits[(size_t)i * ldw + (c >> 5)] >> (c & 31)) & 1u)) continue;
        s += (double)Xf[(size_t)i * ld + c];
        ++cnt;
    }
    const double mu = cnt > 0 ? s / cnt : 0.0;
    double v = 0.0;
    for (int i = 0; i < n; ++i) {
        if (bits && !((bits[(size_t)i * ldw + (c >> 5)] >> (c & 31)) & 1u)) continue;
        const double d = (double)Xf[(size_t)i * ld + c] - mu;
        v += d * d;
    }
    const double sd = cnt > 0 ? sqrt(v / cnt) : 0.0;
    mean[c] = mu;
    scale[c] = sd > 0.0 ? sd : 1.0;
}

// observed entries -> (x - mean) / scale; missing entries and padding stay 0
__global__ void standardize_kernel(float* __restrict__ Xf, double* __restrict__ Xd, const uint32_t* __restrict__ bits,
                                   int n, int p, int ld, int ldw, const double* __restrict__ mean,
                                   const double* __restrict__ scale) {
    const size_t total = (size_t)n * ld;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k / ld), c = (int)(k % ld);
        if (c >= p) continue;
        if (bits && !((bits[(size_t)i * ldw + (c >> 5)] >> (c & 31)) & 1u)) continue;
        const double z = ((double)Xf[k] - mean[c]) / scale[c];
        Xf[k] = (float)z;
        if (Xd) Xd[k] = z;
    }
}

// per-column sum of squared deviations of Y_0 (double), then one fixed-order total
__global__ void centred_ss_kernel(const float* __restrict__ Y0f, const double* __restrict__ Y0d, int n, int p, int ld,
                                  const double* __restrict__ colmean, double* __restrict__ colss) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p) return;
    // mean of Y_0 over all rows equals the observed mean (missing rows hold it)
    const double mu = colmean[c];
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        const double y = Y0d ? Y0d[(size_t)i * ld + c] : (double)Y0f[(size_t)i * ld + c];
        s += (y - mu) * (y - mu);
    }
    colss[c] = s;
}

__global__ void total_kernel(const double* __restrict__ v, int len, double* __restrict__ out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int k = threadIdx.x; k < len; k += blockDim.x) s += v[k];
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) t += red[k];
        *out = t;
    }
}

}  // namespace

cudaError_t launch_pack_input(const float* X, const uint8_t* mask, int64_t n, int64_t p, int64_t ld_in, float* Xf,
                              double* Xd, uint32_t* maskbits, int ld, int ldw, int* bad_count, cudaStream_t s) {
    // bad_count[0]: non-finite observed entries, bad_count[1]: rows with nothing observed
    size_t total = (size_t)n * ld;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    count_launches(1);
    pack_values_kernel<<<blocks, 256, 0, s>>>(X, mask, n, p, ld_in, Xf, Xd, ld, bad_count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !mask) return e;
    count_launches(1);
    pack_mask_kernel<<<(unsigned)n, 128, 0, s>>>(mask, n, p, ld_in, maskbits, ldw, bad_count + 1);
    return cudaGetLastError();
}

cudaError_t launch_standardize(float* Xf, double* Xd, const uint32_t* maskbits, int n, int p, int ld, int ldw,
                               double* work, cudaStream_t s) {
    // work holds 2 * ld doubles: the column means, then the scales
    const int tb = 128;
    count_launches(1);
    column_stats_kernel<<<(p + tb - 1) / tb, tb, 0, s>>>(Xf, maskbits, n, p, ld, ldw, work, work + ld);
    size_t total = (size_t)n * ld;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    count_launches(1);
    standardize_kernel<<<blocks, 256, 0, s>>>(Xf, Xd, maskbits, n, p, ld, ldw, work, work + ld);
    return cudaGetLastError();
}

cudaError_t launch_fill_missing(const float* Xf, const double* Xd, const uint32_t* maskbits, int n, int p, int ld,
                                int ldw, double* colmean, float* Y0f, double* Y0d, double* ss, cudaStream_t s) {
    (void)Xd;
    const int tb = 128;
    count_launches(1);
    column_mean_kernel<<<(p + tb - 1) / tb, tb, 0, s>>>(Xf, maskbits, n, p, ld, ldw, colmean);
    size_t total = (size_t)n * ld;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    count_launches(1);
    fill_kernel<<<blocks, 256, 0, s>>>(Xf, maskbits, n, p, ld, ldw, colmean, Y0f, Y0d);
    // the caller's colmean buffer holds 2 * ld doubles; the second half takes
    // the per-column sums of squared deviations
    double* colss = colmean + ld;
    count_launches(1);
    centred_ss_kernel<<<(p + tb - 1) / tb, tb, 0, s>>>(Y0f, Y0d, n, p, ld, colmean, colss);
    count_launches(1);
    total_kernel<<<1, 1024, 0, s>>>(colss, p, ss);
    return cudaGetLastError();
}

}  // namespace ccx
