// Principal axes of Y_0 and projection of the path onto them (Evaluation of
// Clusters: the cluster path is displayed on principal components of the data;
// projecting on the GPU makes each gamma's output n x q instead of n x p).
//
// Axes by subspace iteration with r = q + 8 vectors: W = Y_c V^T, V = W^T Y_c,
// rows of V orthonormalised (modified Gram-Schmidt, twice), all in double over
// the float rows of Y_0 centred by the double column means; then Rayleigh-Ritz:
// the r x r matrix W^T W is diagonalised by cyclic Jacobi rotations and the
// leading q Ritz vectors are the axes, each signed so that its entry of
// largest magnitude is positive.  Every sum runs in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "ccx_internal.h"

namespace ccx {
namespace {

constexpr int kPcMaxR = 16;
constexpr int kPcThreads = 256;
constexpr int kPcIters = 60;

__device__ double block_sum_d(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// deterministic start vectors in [-1, 1)
__global__ void pc_init_kernel(double* V, int r, int p) {
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= (size_t)r * p) return;
    uint64_t x = t * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    V[t] = (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// W[i][c] = sum_k (y_ik - mean_k) V[c][k]: one warp per row
__global__ void pc_mult_kernel(const float* __restrict__ Y, const double* __restrict__ mean,
                               const double* __restrict__ V, int n, int p, int ld, int r, double* __restrict__ W) {
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double acc[kPcMaxR];
#pragma unroll
    for (int c = 0; c < kPcMaxR; ++c) acc[c] = 0.0;
    for (int k = lane; k < p; k += 32) {
        const double y = (double)Y[(size_t)i * ld + k] - mean[k];
#pragma unroll
        for (int c = 0; c < kPcMaxR; ++c)
            if (c < r) acc[c] += y * V[(size_t)c * p + k];
    }
#pragma unroll
    for (int c = 0; c < kPcMaxR; ++c) {
        if (c >= r) break;
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) W[(size_t)i * r + c] = v;
    }
}

// V[c][k] = sum_i (y_ik - mean_k) W[i][c]: one thread per column
__global__ void pc_multT_kernel(const float* __restrict__ Y, const double* __restrict__ mean,
                                const double* __restrict__ W, int n, int p, int ld, int r, double* __restrict__ V) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p) return;
    double acc[kPcMaxR];
#pragma unroll
    for (int c = 0; c < kPcMaxR; ++c) acc[c] = 0.0;
    const double mk = mean[k];
    for (int i = 0; i < n; ++i) {
        const double y = (double)Y[(size_t)i * ld + k] - mk;
#pragma unroll
        for (int c = 0; c < kPcMaxR; ++c)
            if (c < r) acc[c] += y * W[(size_t)i * r + c];
    }
    for (int c = 0; c < r; ++c) V[(size_t)c * p + k] = acc[c];
}

// orthonormal rows of V (r x p): modified Gram-Schmidt, applied twice; one block
__global__ void pc_orth_kernel(double* V, int r, int p) {
    __shared__ double red[33];
    for (int pass = 0; pass < 2; ++pass)
        for (int c = 0; c < r; ++c) {
            double* vc = V + (size_t)c * p;
            for (int d = 0; d < c; ++d) {
                const double* vd = V + (size_t)d * p;
                double s = 0.0;
                for (int k = threadIdx.x; k < p; k += blockDim.x) s += vc[k] * vd[k];
                const double dot = block_sum_d(s, red);
                for (int k = threadIdx.x; k < p; k += blockDim.x) vc[k] -= dot * vd[k];
                __syncthreads();
            }
            double s = 0.0;
            for (int k = threadIdx.x; k < p; k += blockDim.x) s += vc[k] * vc[k];
            const double nrm = sqrt(block_sum_d(s, red));
            const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
            for (int k = threadIdx.x; k < p; k += blockDim.x) vc[k] *= inv;
            __syncthreads();
        }
}

// B = W^T W (r x r); one block
__global__ void pc_small_gram_kernel(const double* __restrict__ W, int n, int r, double* __restrict__ B) {
    __shared__ double red[33];
    for (int a = 0; a < r; ++a)
        for (int b = a; b < r; ++b) {
            double s = 0.0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) s += W[(size_t)i * r + a] * W[(size_t)i * r + b];
            const double v = block_sum_d(s, red);
            if (threadIdx.x == 0) {
                B[a * r + b] = v;
                B[b * r + a] = v;
            }
        }
}

// Eigen-decomposition of the symmetric r x r matrix B by cyclic Jacobi
// rotations (one thread); E columns = eigenvectors, sorted by eigenvalue,
// largest first.
__global__ void pc_jacobi_kernel(double* B, int r, double* E, double* lam) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) E[a * r + b] = (a == b) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int a = 0; a < r; ++a)
            for (int b = 0; b < r; ++b) {
                const double v = B[a * r + b] * B[a * r + b];
                tot += v;
                if (a != b) off += v;
            }
        if (off <= 1e-30 * tot) break;
        for (int a = 0; a < r - 1; ++a)
            for (int b = a + 1; b < r; ++b) {
                const double bab = B[a * r + b];
                if (bab == 0.0) continue;
                // rotation in the (a, b) plane that zeroes B_ab
                const double theta = (B[b * r + b] - B[a * r + a]) / (2.0 * bab);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < r; ++k) {
                    const double bka = B[k * r + a], bkb = B[k * r + b];
                    B[k * r + a] = c * bka - s * bkb;
                    B[k * r + b] = s * bka + c * bkb;
                }
                for (int k = 0; k < r; ++k) {
                    const double bak = B[a * r + k], bbk = B[b * r + k];
                    B[a * r + k] = c * bak - s * bbk;
                    B[b * r + k] = s * bak + c * bbk;
                }
                for (int k = 0; k < r; ++k) {
                    const double eka = E[k * r + a], ekb = E[k * r + b];
                    E[k * r + a] = c * eka - s * ekb;
                    E[k * r + b] = s * eka + c * ekb;
                }
            }
    }
    for (int a = 0; a < r; ++a) lam[a] = B[a * r + a];
    // selection sort of the eigenpairs, largest eigenvalue first
    for (int a = 0; a < r; ++a) {
        int best = a;
        for (int b = a + 1; b < r; ++b)
            if (lam[b] > lam[best]) best = b;
        if (best != a) {
            const double t = lam[a];
            lam[a] = lam[best];
            lam[best] = t;
            for (int k = 0; k < r; ++k) {
                const double u = E[k * r + a];
                E[k * r + a] = E[k * r + best];
                E[k * r + best] = u;
            }
        }
    }
}

// axes[c][k] = sum_a E[a][c] V[a][k] for c < q
__global__ void pc_rotate_kernel(const double* __restrict__ V, const double* __restrict__ E, int r, int p, int q,
                                 double* __restrict__ axes) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p) return;
    for (int c = 0; c < q; ++c) {
        double s = 0.0;
        for (int a = 0; a < r; ++a) s += E[a * r + c] * V[(size_t)a * p + k];
        axes[(size_t)c * p + k] = s;
    }
}

// sign rule: the entry of largest magnitude (first on ties) of each axis is positive; one block per axis
__global__ void pc_sign_kernel(double* axes, int p) {
    double* a = axes + (size_t)blockIdx.x * p;
    __shared__ double bv[kPcThreads];
    __shared__ int bi[kPcThreads];
    double best = -1.0;
    int idx = 0x7fffffff;
    for (int k = threadIdx.x; k < p; k += blockDim.x) {
        const double v = fabs(a[k]);
        if (v > best) {
            best = v;
            idx = k;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double v2 = bv[threadIdx.x + s];
            const int i2 = bi[threadIdx.x + s];
            if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
                bv[threadIdx.x] = v2;
                bi[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    const bool flip = a[bi[0]] < 0.0;
    __syncthreads();
    if (flip)
        for (int k = threadIdx.x; k < p; k += blockDim.x) a[k] = -a[k];
}

// S[i][c] = sum_k (u_ik - mean_k) axes[c][k]: one warp per row
__global__ void pc_project_kernel(const float* __restrict__ U, int ldu, const double* __restrict__ mean,
                                  const double* __restrict__ axes, int n, int p, int q, float* __restrict__ S) {
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double acc[kPcMaxR];
#pragma unroll
    for (int c = 0; c < kPcMaxR; ++c) acc[c] = 0.0;
    for (int k = lane; k < p; k += 32) {
        const double u = (double)U[(size_t)i * ldu + k] - mean[k];
#pragma unroll
        for (int c = 0; c < kPcMaxR; ++c)
            if (c < q) acc[c] += u * axes[(size_t)c * p + k];
    }
#pragma unroll
    for (int c = 0; c < kPcMaxR; ++c) {
        if (c >= q) break;
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) S[(size_t)i * q + c] = (float)v;
    }
}

}  // namespace

int pc_max_axes() { return kPcMaxR - 8; }

cudaError_t pc_axes(const float* Y0f, const double* mean, int n, int p, int ld, int q, double* axes, double* var_h,
                    cudaStream_t s) {
    if (q < 1 || q > kPcMaxR - 8) return cudaErrorInvalidValue;
    const int r = std::min(q + 8, std::min(n, p));
    if (r < q) return cudaErrorInvalidValue;
    double *V = nullptr, *W = nullptr, *B = nullptr, *E = nullptr, *lam = nullptr;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        cudaFree(V);
        cudaFree(W);
        cudaFree(B);
        cudaFree(E);
        cudaFree(lam);
    };
    if ((e = cudaMalloc(&V, sizeof(double) * (size_t)r * p)) != cudaSuccess) return cleanup(), e;
    if ((e = cudaMalloc(&W, sizeof(double) * (size_t)n * r)) != cudaSuccess) return cleanup(), e;
    if ((e = cudaMalloc(&B, sizeof(double) * r * r)) != cudaSuccess) return cleanup(), e;
    if ((e = cudaMalloc(&E, sizeof(double) * r * r)) != cudaSuccess) return cleanup(), e;
    if ((e = cudaMalloc(&lam, sizeof(double) * r)) != cudaSuccess) return cleanup(), e;
    const int rows_per_block = kPcThreads / 32;
    const dim3 g_rows((n + rows_per_block - 1) / rows_per_block), g_cols((p + kPcThreads - 1) / kPcThreads);
    count_launches(2);
    pc_init_kernel<<<(int)(((size_t)r * p + kPcThreads - 1) / kPcThreads), kPcThreads, 0, s>>>(V, r, p);
    pc_orth_kernel<<<1, 1024, 0, s>>>(V, r, p);
    for (int it = 0; it < kPcIters; ++it) {
        count_launches(3);
        pc_mult_kernel<<<g_rows, kPcThreads, 0, s>>>(Y0f, mean, V, n, p, ld, r, W);
        pc_multT_kernel<<<g_cols, kPcThreads, 0, s>>>(Y0f, mean, W, n, p, ld, r, V);
        pc_orth_kernel<<<1, 1024, 0, s>>>(V, r, p);
    }
    count_launches(5);
    pc_mult_kernel<<<g_rows, kPcThreads, 0, s>>>(Y0f, mean, V, n, p, ld, r, W);
    pc_small_gram_kernel<<<1, kPcThreads, 0, s>>>(W, n, r, B);
    pc_jacobi_kernel<<<1, 32, 0, s>>>(B, r, E, lam);
    pc_rotate_kernel<<<g_cols, kPcThreads, 0, s>>>(V, E, r, p, q, axes);
    pc_sign_kernel<<<q, kPcThreads, 0, s>>>(axes, p);
    if ((e = cudaGetLastError()) != cudaSuccess) return cleanup(), e;
    std::vector<double> hl(r);
    if ((e = cudaMemcpyAsync(hl.data(), lam, sizeof(double) * r, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cleanup(), e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cleanup(), e;
    for (int c = 0; c < q; ++c) var_h[c] = hl[c] / n;
    cleanup();
    return cudaSuccess;
}

cudaError_t pc_project(const float* U, int ldu, const double* mean, const double* axes, int n, int p, int q, float* S,
                       cudaStream_t s) {
    const int rows_per_block = kPcThreads / 32;
    count_launches(1);
    pc_project_kernel<<<(n + rows_per_block - 1) / rows_per_block, kPcThreads, 0, s>>>(U, ldu, mean, axes, n, p, q,
                                                                                        S);
    return cudaGetLastError();
}

}  // namespace ccx
