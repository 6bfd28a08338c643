// kNN union graph with Gaussian-kernel weights (Calibration of Weights, Eq. 8).
//
// 1. y_i = row i of Y_0 (missing entries at the observed column mean, in
//    double); sq_i = ||y_i||^2 and nrm_i = ||y_i|| in double.
// 2. Gram matrix G ~ Y Y^T of the float copy of Y_0 (gram_f32_kernel, or the
//    tensor-core kernel in gram_tc.cu), giving approximate squared distances
//    a_ij = sq_i + sq_j - 2 G_ij.
// 3. Per row i (knn_row_kernel): with a rigorous per-pair bound
//    |a_ij - d2_ij| <= b_ij, T = k-th smallest (a_ij + b_ij) bounds the true
//    k-th smallest distance from above, so every true neighbour satisfies
//    a_ij - b_ij <= T.  Those candidates get their distance recomputed
//    exactly from the rows (double differences and sums in a fixed order),
//    and the k smallest by (d2, j) are kept: ties go to the smaller index.
// 4. The union i ~_k j, phi, the weights and the normalisation are formed on
//    the device from the exact d2 (knn_weights.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <set>
#include <string>
#include <vector>

#include "ccx_internal.h"

namespace ccx {

// defined in gram_tc.cu: G = Y Y^T on the tensor cores; returns cudaErrorNotSupported
// when the shape is outside the kernel's tiling, and the per-entry relative
// input rounding it used through *unit.
cudaError_t launch_gram_tc(const float* Y, int n, int p, int ld, float* G, double* unit, cudaStream_t s, int bf16);

namespace {

constexpr int kRowThreads = 256;

__global__ void row_norm_kernel(const float* __restrict__ Xf, const uint32_t* __restrict__ bits,
                                const double* __restrict__ colmean, int n, int p, int ld, int ldw,
                                double* __restrict__ sq) {
    const int i = blockIdx.x;
    __shared__ double red[32];
    double s = 0.0;
    for (int c = threadIdx.x; c < p; c += blockDim.x) {
        const bool obs = bits ? ((bits[(size_t)i * ldw + (c >> 5)] >> (c & 31)) & 1u) : true;
        const double y = obs ? (double)Xf[(size_t)i * ld + c] : colmean[c];
        s += y * y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        sq[i] = t;
    }
}

// Plain FP32 Gram, 64 x 64 tiles, 16 x 16 threads, 4 x 4 outputs each.
__global__ void __launch_bounds__(256) gram_f32_kernel(const float* __restrict__ Y, int n, int p, int ld,
                                                       float* __restrict__ G) {
    __shared__ float sa[16][64 + 4];
    __shared__ float sb[16][64 + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < p; k0 += 16) {
        for (int q = threadIdx.x; q < 64 * 16; q += 256) {
            const int r = q >> 4, kk = q & 15;
            const int gr = row0 + r, gc = col0 + r, gk = k0 + kk;
            sa[kk][r] = (gr < n && gk < p) ? Y[(size_t)gr * ld + gk] : 0.f;
            sb[kk][r] = (gc < n && gk < p) ? Y[(size_t)gc * ld + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = sa[kk][ty * 4 + u];
                b[u] = sb[kk][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = row0 + ty * 4 + u, c = col0 + tx * 4 + v;
            if (r < n && c < n) G[(size_t)r * n + c] = acc[u][v];
        }
}

// bitonic sort of (key, idx) pairs in shared memory, ascending by (key, idx)
__device__ void bitonic_sort(double* key, int* idx, int len_pow2) {
    for (int size = 2; size <= len_pow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < len_pow2; t += blockDim.x) {
                const int partner = t ^ stride;
                if (partner > t) {
                    const bool up = ((t & size) == 0);
                    const double ka = key[t], kb = key[partner];
                    const int ia = idx[t], ib = idx[partner];
                    const bool gt = (ka > kb) || (ka == kb && ia > ib);
                    if (gt == up) {
                        key[t] = kb;
                        key[partner] = ka;
                        idx[t] = ib;
                        idx[partner] = ia;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Geographic distance in degrees between (latitude, longitude) pairs in
// degrees: the coordinate difference with longitude modulo 360 (Calibration of
// Weights), or the great-circle angle from the spherical case of Vincenty's
// formula (atan2 of the cross and dot products; accurate up to antipodes).
__device__ double geo_deg(const double* __restrict__ geo, int i, int j, int geodesic) {
    const double lat1 = geo[2 * i], lon1 = geo[2 * i + 1], lat2 = geo[2 * j], lon2 = geo[2 * j + 1];
    if (!geodesic) {
        double dl = fmod(fabs(lon1 - lon2), 360.0);
        if (dl > 180.0) dl = 360.0 - dl;
        const double dp = lat1 - lat2;
        return sqrt(dp * dp + dl * dl);
    }
    const double r = 3.14159265358979323846 / 180.0;
    const double p1 = lat1 * r, p2 = lat2 * r, dl = (lon2 - lon1) * r;
    const double y = hypot(cos(p2) * sin(dl), cos(p1) * sin(p2) - sin(p1) * cos(p2) * cos(dl));
    const double x = sin(p1) * sin(p2) + cos(p1) * cos(p2) * cos(dl);
    return atan2(y, x) / r;
}

__global__ void __launch_bounds__(kRowThreads) knn_row_kernel(
    const float* __restrict__ Xf, const uint32_t* __restrict__ bits, const double* __restrict__ colmean,
    const double* __restrict__ sq, const float* __restrict__ G, double gunit, int use_all, int n, int p, int ld,
    int ldw, int k, int npow2, int* __restrict__ nbr, double* __restrict__ nd2, const double* __restrict__ geo,
    double alpha, int geodesic) {
    extern __shared__ __align__(16) unsigned char sm[];
    double* key = reinterpret_cast<double*>(sm);          // npow2
    double* av = key + npow2;                             // n: lower bound of the distance key
    double* bv = av + n;                                  // n: upper bound of the distance key
    int* idx = reinterpret_cast<int*>(bv + n);            // npow2
    int* cand = idx + npow2;                              // n
    __shared__ int ncand;
    __shared__ double Tsh;
    const int i = blockIdx.x;
    const double sqi = sq[i], nri = sqrt(sq[i]);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        if (use_all) {
            av[j] = 0.0;
            bv[j] = 0.0;
        } else {
            const double a = sqi + sq[j] - 2.0 * (double)G[(size_t)i * n + j];
            // |G_ij - <y_i, y_j>| <= gunit * ||y_i|| ||y_j||; d2 = sq_i + sq_j - 2 <y_i, y_j>
            const double b = 2.0 * gunit * nri * sqrt(sq[j]) * (1.0 + 1e-9) + 1e-300;
            if (geo) {
                // composite key alpha ||y_i - y_j|| + (1 - alpha) g_ij, g exact in double
                const double g = (1.0 - alpha) * geo_deg(geo, i, j, geodesic);
                av[j] = (alpha * sqrt(fmax(a - b, 0.0)) + g) * (1.0 - 1e-12);
                bv[j] = (alpha * sqrt(fmax(a + b, 0.0)) + g) * (1.0 + 1e-12) + 1e-300;
            } else {
                av[j] = a - b;      // squared-distance key
                bv[j] = a + b;
            }
        }
    }
    __syncthreads();
    if (use_all) {
        if (threadIdx.x == 0) Tsh = INFINITY;
    } else {
        for (int t = threadIdx.x; t < npow2; t += blockDim.x) {
            key[t] = (t < n && t != i) ? bv[t] : INFINITY;
            idx[t] = t;
        }
        __syncthreads();
        bitonic_sort(key, idx, npow2);
        if (threadIdx.x == 0) Tsh = key[k - 1];
    }
    if (threadIdx.x == 0) ncand = 0;
    __syncthreads();
    const double T = Tsh;
    // candidates: lower bound <= T (order fixed later by the sort)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        if (j != i && (use_all || av[j] <= T)) {
            const int slot = atomicAdd(&ncand, 1);
            cand[slot] = j;
        }
    }
    __syncthreads();
    const int nc = ncand;
    // exact distances, one warp per candidate, double throughout
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = wid; q < nc; q += nw) {
        const int j = cand[q];
        double s = 0.0;
        for (int c = lane; c < p; c += 32) {
            const uint32_t wi = bits ? bits[(size_t)i * ldw + (c >> 5)] : 0xffffffffu;
            const uint32_t wj = bits ? bits[(size_t)j * ldw + (c >> 5)] : 0xffffffffu;
            const double yi = ((wi >> (c & 31)) & 1u) ? (double)Xf[(size_t)i * ld + c] : colmean[c];
            const double yj = ((wj >> (c & 31)) & 1u) ? (double)Xf[(size_t)j * ld + c] : colmean[c];
            const double dd = yi - yj;
            s += dd * dd;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        // av now holds the exact key of each candidate: d2, or the composite distance
        if (lane == 0) av[j] = geo ? alpha * sqrt(s) + (1.0 - alpha) * geo_deg(geo, i, j, geodesic) : s;
    }
    __syncthreads();
    int cp2 = 1;
    while (cp2 < nc) cp2 <<= 1;
    for (int t = threadIdx.x; t < cp2; t += blockDim.x) {
        if (t < nc) {
            key[t] = av[cand[t]];
            idx[t] = cand[t];
        } else {
            key[t] = INFINITY;
            idx[t] = 0x7fffffff;
        }
    }
    __syncthreads();
    bitonic_sort(key, idx, cp2);
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        nbr[(size_t)i * k + r] = idx[r];
        nd2[(size_t)i * k + r] = geo ? key[r] * key[r] : key[r];   // squared distance for the weights
    }
}

__global__ void edge_d2_kernel(const float* __restrict__ Y, int p, int ld, const int* __restrict__ ei,
                               const int* __restrict__ ej, int m, double* __restrict__ d2) {
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
    if (lane == 0) d2[e] = s;
}

}  // namespace

cudaError_t edge_distances(const float* Y0f, int n, int p, int ld, const int* ei_d, const int* ej_d, int m,
                           double* d2_d, cudaStream_t s) {
    (void)n;
    if (m == 0) return cudaSuccess;
    count_launches(1);
    edge_d2_kernel<<<(m + 7) / 8, 256, 0, s>>>(Y0f, p, ld, ei_d, ej_d, m, d2_d);
    return cudaGetLastError();
}

// Y0f: float Y_0 (device, n x ld); the knn needs the exact rows as well, which
// are Xf + mask + colmean.  Those are passed through knn_args (set by the API).
struct KnnDeviceArgs {
    const float* Xf;
    const uint32_t* bits;
    const double* colmean;
    int ldw;
};
static thread_local KnnDeviceArgs g_knn_args;
void knn_set_exact_rows(const float* Xf, const uint32_t* bits, const double* colmean, int ldw) {
    g_knn_args = {Xf, bits, colmean, ldw};
}

// The k nearest neighbours of every row on the device: nbr (n x kk) and their
// exact squared distances nd2, each row ascending by (d2, j).  The caller frees
// *nbr and *nd2.
static cudaError_t knn_lists(const float* Y0f, int n, int p, int ld, int kk, cudaStream_t s, int** nbr_out,
                             double** nd2_out, const double* geo = nullptr, double alpha = 1.0, int geodesic = 0,
                             int gram = 0) {
    const KnnDeviceArgs ka = g_knn_args;
    const int use_all = (kk >= n - 1) ? 1 : 0;
    cudaError_t e;
    double* sq = nullptr;
    float* G = nullptr;
    int* nbr = nullptr;
    double* nd2 = nullptr;
    double gunit = 0.0;
    auto cleanup = [&]() {
        cudaFree(sq);
        cudaFree(G);
        cudaFree(nbr);
        cudaFree(nd2);
    };
    if ((e = cudaMalloc(&sq, sizeof(double) * n)) != cudaSuccess) return cleanup(), e;
    if ((e = cudaMalloc(&nbr, sizeof(int) * (size_t)n * kk)) != cudaSuccess) return cleanup(), e;
    if ((e = cudaMalloc(&nd2, sizeof(double) * (size_t)n * kk)) != cudaSuccess) return cleanup(), e;
    count_launches(1);
    row_norm_kernel<<<n, 256, 0, s>>>(ka.Xf, ka.bits, ka.colmean, n, p, ld, ka.ldw, sq);
    if ((e = cudaGetLastError()) != cudaSuccess) return cleanup(), e;
    if (!use_all) {
        if ((e = cudaMalloc(&G, sizeof(float) * (size_t)n * n)) != cudaSuccess) return cleanup(), e;
        e = gram == 2 ? cudaErrorNotSupported : launch_gram_tc(Y0f, n, p, ld, G, &gunit, s, gram == 1 ? 1 : 0);
        if (e == cudaErrorNotSupported) {
            (void)cudaGetLastError();
            dim3 grid((n + 63) / 64, (n + 63) / 64);
            count_launches(1);
            gram_f32_kernel<<<grid, 256, 0, s>>>(Y0f, n, p, ld, G);
            e = cudaGetLastError();
            // float inputs carry the float rounding of the filled missing entries
            // (relative 2^-24) and FP32 accumulation over p terms
            const double u = 1.0 / 16777216.0;
            gunit = 2.0 * u + (double)(p + 2) * u;
        }
        if (e != cudaSuccess) return cleanup(), e;
    }
    int npow2 = 1;
    while (npow2 < n) npow2 <<= 1;
    const size_t smem = sizeof(double) * (size_t)(npow2 + 2 * n) + sizeof(int) * (size_t)(npow2 + n);
    if ((e = cudaFuncSetAttribute(knn_row_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return cleanup(), e;
    count_launches(1);
    knn_row_kernel<<<n, kRowThreads, smem, s>>>(ka.Xf, ka.bits, ka.colmean, sq, G, gunit, use_all, n, p, ld, ka.ldw,
                                                kk, npow2, nbr, nd2, geo, alpha, geodesic);
    if ((e = cudaGetLastError()) != cudaSuccess) return cleanup(), e;
    cudaFree(sq);
    cudaFree(G);
    *nbr_out = nbr;
    *nd2_out = nd2;
    return cudaSuccess;
}

// edges (i, nbr[i][r]) for r < k of the neighbour lists (kk per row)
__global__ void probe_edges_kernel(const int* __restrict__ nbr, int n, int kk, int k, int* __restrict__ ei,
                                   int* __restrict__ ej) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * k) return;
    const int i = q / k, r = q - i * k;
    ei[q] = i;
    ej[q] = nbr[(size_t)i * kk + r];
}

__global__ void fill_ones_kernel(uint8_t* f, int m) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < m) f[q] = 1;
}

cudaError_t knn_min_connected_k(const float* Y0f, int n, int p, int ld, int k_max, cudaStream_t s, int* k_out,
                                int* probes, std::string* err) {
    *k_out = 0;
    *probes = 0;
    if (n > 4096) {
        *err = "kNN build supports n <= 4096 in this build";
        return cudaErrorNotSupported;
    }
    const int kk = std::min(k_max, n - 1);
    if (kk <= 0) return cudaSuccess;
    int* nbr = nullptr;
    double* nd2 = nullptr;
    cudaError_t e = knn_lists(Y0f, n, p, ld, kk, s, &nbr, &nd2);
    if (e != cudaSuccess) return e;
    const size_t mmax = (size_t)n * kk;
    int *ei = nullptr, *ej = nullptr, *lab = nullptr, *scratch = nullptr, *ncl = nullptr;
    uint8_t* ones = nullptr;
    auto cleanup = [&]() {
        cudaFree(nbr);
        cudaFree(nd2);
        cudaFree(ei);
        cudaFree(ej);
        cudaFree(lab);
        cudaFree(scratch);
        cudaFree(ncl);
        cudaFree(ones);
    };
    if ((e = cudaMalloc(&ei, sizeof(int) * mmax)) != cudaSuccess) return cleanup(), e;
    if ((e = cudaMalloc(&ej, sizeof(int) * mmax)) != cudaSuccess) return cleanup(), e;
    if ((e = cudaMalloc(&ones, mmax)) != cudaSuccess) return cleanup(), e;
    if ((e = cudaMalloc(&lab, sizeof(int) * n)) != cudaSuccess) return cleanup(), e;
    if ((e = cudaMalloc(&scratch, sizeof(int) * n)) != cudaSuccess) return cleanup(), e;
    if ((e = cudaMalloc(&ncl, sizeof(int))) != cudaSuccess) return cleanup(), e;
    count_launches(1);
    fill_ones_kernel<<<(int)((mmax + 255) / 256), 256, 0, s>>>(ones, (int)mmax);
    if ((e = cudaGetLastError()) != cudaSuccess) return cleanup(), e;
    // the union graph only grows with k, so its connectivity is monotone in k: bisection
    auto connected = [&](int k, bool* yes) -> cudaError_t {
        const int m = n * k;
        count_launches(1);
        probe_edges_kernel<<<(m + 255) / 256, 256, 0, s>>>(nbr, n, kk, k, ei, ej);
        cudaError_t r = cudaGetLastError();
        if (r == cudaSuccess) r = launch_fused_labels(n, m, ei, ej, ones, lab, ncl, scratch, s);
        int h = 0;
        if (r == cudaSuccess) r = cudaMemcpyAsync(&h, ncl, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (r == cudaSuccess) r = cudaStreamSynchronize(s);
        if (r == cudaSuccess && h < 0) r = cudaErrorUnknown;   // components did not settle
        *yes = (h == 1);
        ++*probes;
        return r;
    };
    bool yes = false;
    if ((e = connected(kk, &yes)) != cudaSuccess) return cleanup(), e;
    if (!yes) return cleanup(), cudaSuccess;
    int lo = 1, hi = kk;   // connected at hi
    while (lo < hi) {
        const int mid = lo + (hi - lo) / 2;
        if ((e = connected(mid, &yes)) != cudaSuccess) return cleanup(), e;
        if (yes) hi = mid;
        else lo = mid + 1;
    }
    *k_out = hi;
    cleanup();
    return cudaSuccess;
}

cudaError_t knn_build(const float* Y0f, int n, int p, int ld, int k, double phi, int phi_auto, int normalize,
                      cudaStream_t s, KnnResult* out, std::string* err, const double* geo, double alpha,
                      int geodesic, int gram) {
    if (n > 4096) {
        *err = "kNN build supports n <= 4096 in this build";
        return cudaErrorNotSupported;
    }
    const int kk = std::min(k, n - 1);
    out->ei.clear();
    out->ej.clear();
    out->w.clear();
    out->d2.clear();
    if (kk <= 0) return cudaSuccess;
    int* nbr = nullptr;
    double* nd2 = nullptr;
    cudaError_t e = knn_lists(Y0f, n, p, ld, kk, s, &nbr, &nd2, geo, alpha, geodesic, gram);
    if (e != cudaSuccess) return e;
    auto cleanup = [&]() {
        cudaFree(nbr);
        cudaFree(nd2);
    };
    e = knn_union_weights(nbr, nd2, n, kk, phi, phi_auto, normalize, s, out);
    cleanup();
    return e;
}

}  // namespace ccx
