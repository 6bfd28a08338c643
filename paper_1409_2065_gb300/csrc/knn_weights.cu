// Union of the k-nearest-neighbour lists and the Gaussian-kernel weights of
// Calibration of Weights, Eq. 8, formed on the device from the lists that
// knn_kernels.cu builds (each row's kk neighbours with their exact squared
// distances):
//   * union i ~_k j: every list entry (i, j) sets bit max(i, j) of row
//     min(i, j) of an n x ceil(n / 32) bitmap.  The edges are the set bits in
//     (row, bit) order, so they come out sorted by (ei, ej) with no sort.  The
//     squared distance of an edge is read from a dense n x n table, written
//     first from the entries with i > j and then from those with i < j, so
//     where both lists hold the pair the smaller endpoint's value is kept.
//   * phi (automatic rule) = 1 / median of d2 over the union edges (0 when
//     that median is 0).  The median is found by a radix select over the bit
//     patterns of the non-negative doubles, whose order is their numeric order.
//   * w = exp(-phi (d2 - min d2)) / sum (normalised rule) or exp(-phi d2).  The
//     sum is taken in a fixed order (each block's grid-strided share, a tree in
//     the block, then the blocks in order), so repeated builds agree bit for bit.
// Edges whose weight underflows to zero are left in; installing an edge set
// drops zero weights.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "ccx_internal.h"

namespace ccx {
namespace {

constexpr int kWThreads = 256;
constexpr int kWMaxBlocks = 1024;

struct KnnScalars {
    unsigned long long prefix, mask;  // radix select: digits fixed so far
    long long kth;                    // rank still sought among keys matching prefix
    unsigned int hist[256];
    unsigned long long dmin_key;      // min over d2 of its key
    double v[2];                      // selected order statistics
    double phi;
    double tot;
};

// order-preserving key of a non-negative double (-0 and +0 both map to 0)
__device__ __forceinline__ unsigned long long d2_key(double d) {
    return d > 0.0 ? (unsigned long long)__double_as_longlong(d) : 0ULL;
}

__global__ void union_mark_kernel(const int* __restrict__ nbr, const double* __restrict__ nd2, int n, int kk,
                                  int W, int from_larger, uint32_t* __restrict__ bits, double* __restrict__ D) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)n * kk) return;
    const int i = (int)(q / kk), j = nbr[q];
    // from_larger: the entries listed by the larger endpoint (i > j); else those with i < j
    if ((i > j) != (from_larger != 0)) return;
    const int a = min(i, j), b = max(i, j);
    D[(size_t)a * n + b] = nd2[q];
    atomicOr(&bits[(size_t)a * W + (b >> 5)], 1u << (b & 31));
}

// one warp per row: the number of union edges (a, b > a) of row a
__global__ void union_count_kernel(const uint32_t* __restrict__ bits, int n, int W, int* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (a >= n) return;
    int c = 0;
    for (int w = lane; w < W; w += 32) c += __popc(bits[(size_t)a * W + w]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[a] = c;
}

// exclusive scan of cnt[0..n) into off[0..n], one block of 1024 threads (n <= 4096)
__global__ void union_scan_kernel(const int* __restrict__ cnt, int n, int* __restrict__ off) {
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b0 = min(n, tid * per), b1 = min(n, b0 + per);
    int s = 0;
    for (int k = b0; k < b1; ++k) s += cnt[k];
    int incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        wsum[lane] = v;   // inclusive over warps
    }
    __syncthreads();
    int run = (warp > 0 ? wsum[warp - 1] : 0) + incl - s;
    for (int k = b0; k < b1; ++k) {
        off[k] = run;
        run += cnt[k];
    }
    if (tid == blockDim.x - 1) off[n] = run;
}

// one warp per row a: its edges (a, b) in increasing b, at off[a] ...
__global__ void union_emit_kernel(const uint32_t* __restrict__ bits, const int* __restrict__ off,
                                  const double* __restrict__ D, int n, int W, int* __restrict__ ei,
                                  int* __restrict__ ej, double* __restrict__ d2) {
    const int lane = threadIdx.x & 31;
    const int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (a >= n) return;
    int base = off[a];
    for (int w0 = 0; w0 < W; w0 += 32) {
        const int w = w0 + lane;
        uint32_t word = w < W ? bits[(size_t)a * W + w] : 0u;
        const int c = __popc(word);
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int pos = base + incl - c;
        while (word) {
            const int b = w * 32 + (__ffs(word) - 1);
            word &= word - 1u;
            ei[pos] = a;
            ej[pos] = b;
            d2[pos] = D[(size_t)a * n + b];
            ++pos;
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
}

__global__ void scalars_init_kernel(KnnScalars* s, long long kth) {
    s->prefix = 0ULL;
    s->mask = 0ULL;
    s->kth = kth;
    for (int d = 0; d < 256; ++d) s->hist[d] = 0u;
}

// histogram of the next 8-bit digit (at `shift`) over the keys that match the digits fixed so far;
// also the minimum key (first pass only)
__global__ void select_hist_kernel(const double* __restrict__ d2, int m, KnnScalars* s, int shift, int with_min) {
    __shared__ unsigned int h[256];
    __shared__ unsigned long long kmin[kWThreads / 32];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0u;
    __syncthreads();
    const unsigned long long prefix = s->prefix, mask = s->mask;
    unsigned long long mn = ~0ULL;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
        const unsigned long long key = d2_key(d2[e]);
        if (key < mn) mn = key;
        if ((key & mask) == prefix) atomicAdd(&h[(unsigned)(key >> shift) & 255u], 1u);
    }
    if (with_min) {
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, mn, o);
            if (y < mn) mn = y;
        }
        if ((threadIdx.x & 31) == 0) kmin[threadIdx.x >> 5] = mn;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        if (h[t]) atomicAdd(&s->hist[t], h[t]);
    if (with_min && threadIdx.x == 0) {
        unsigned long long b = ~0ULL;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) b = kmin[k] < b ? kmin[k] : b;
        atomicMin(&s->dmin_key, b);
    }
}

// fixes the digit at `shift` holding rank kth; at the last digit stores the value in v[slot]
__global__ void select_pick_kernel(KnnScalars* s, int shift, int slot) {
    const long long kth = s->kth;
    unsigned long long below = 0ULL;
    int dg = 255;
    for (int d = 0; d < 256; ++d) {
        if ((long long)(below + s->hist[d]) > kth) {
            dg = d;
            break;
        }
        below += s->hist[d];
    }
    s->kth = kth - (long long)below;
    s->prefix |= (unsigned long long)dg << shift;
    s->mask |= 255ULL << shift;
    for (int d = 0; d < 256; ++d) s->hist[d] = 0u;
    if (shift == 0) s->v[slot] = __longlong_as_double((long long)s->prefix);
}

__global__ void phi_kernel(KnnScalars* s, int m, double phi, int phi_auto) {
    if (phi_auto) {
        const double med = (m & 1) ? s->v[0] : 0.5 * (s->v[0] + s->v[1]);
        phi = med > 0.0 ? 1.0 / med : 0.0;
    }
    s->phi = phi;
}

// w = exp(-phi (d2 - dmin)) (normalised) or exp(-phi d2); per-block sums of w into part[]
__global__ void weight_kernel(const double* __restrict__ d2, int m, const KnnScalars* s, int normalize,
                              double* __restrict__ w, double* __restrict__ part) {
    __shared__ double red[kWThreads / 32];
    const double phi = s->phi;
    const double dmin = normalize ? __longlong_as_double((long long)s->dmin_key) : 0.0;
    double acc = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
        const double v = exp(-phi * (d2[e] - dmin));
        w[e] = v;
        acc += v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        part[blockIdx.x] = t;
    }
}

__global__ void weight_total_kernel(const double* __restrict__ part, int nb, KnnScalars* s) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[b];
    s->tot = t;
}

__global__ void weight_scale_kernel(double* __restrict__ w, int m, const KnnScalars* s) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) w[e] /= s->tot;
}

}  // namespace

cudaError_t knn_union_weights(const int* nbr, const double* nd2, int n, int kk, double phi, int phi_auto,
                              int normalize, cudaStream_t s, KnnResult* out) {
    const int W = (n + 31) / 32;
    uint32_t* bits = nullptr;
    double* D = nullptr;
    int *cnt = nullptr, *off = nullptr, *ei = nullptr, *ej = nullptr;
    double *d2 = nullptr, *w = nullptr, *part = nullptr;
    KnnScalars* sc = nullptr;
    auto cleanup = [&]() {
        cudaFree(bits);
        cudaFree(D);
        cudaFree(cnt);
        cudaFree(off);
        cudaFree(ei);
        cudaFree(ej);
        cudaFree(d2);
        cudaFree(w);
        cudaFree(part);
        cudaFree(sc);
    };
    cudaError_t e;
#define KW_TRY(x)                        \
    do {                                 \
        if ((e = (x)) != cudaSuccess) {  \
            cleanup();                   \
            return e;                    \
        }                                \
    } while (0)
    KW_TRY(cudaMalloc(&bits, sizeof(uint32_t) * (size_t)n * W));
    KW_TRY(cudaMalloc(&D, sizeof(double) * (size_t)n * n));
    KW_TRY(cudaMalloc(&cnt, sizeof(int) * (size_t)n));
    KW_TRY(cudaMalloc(&off, sizeof(int) * (size_t)(n + 1)));
    KW_TRY(cudaMalloc(&part, sizeof(double) * kWMaxBlocks));
    KW_TRY(cudaMalloc(&sc, sizeof(KnnScalars)));
    KW_TRY(cudaMemsetAsync(bits, 0, sizeof(uint32_t) * (size_t)n * W, s));
    KW_TRY(cudaMemsetAsync(&sc->dmin_key, 0xff, sizeof(unsigned long long), s));
    const long long entries = (long long)n * kk;
    const int mark_blocks = (int)((entries + kWThreads - 1) / kWThreads);
    const int row_blocks = (n + kWThreads / 32 - 1) / (kWThreads / 32);
    count_launches(4);
    union_mark_kernel<<<mark_blocks, kWThreads, 0, s>>>(nbr, nd2, n, kk, W, 1, bits, D);
    union_mark_kernel<<<mark_blocks, kWThreads, 0, s>>>(nbr, nd2, n, kk, W, 0, bits, D);
    union_count_kernel<<<row_blocks, kWThreads, 0, s>>>(bits, n, W, cnt);
    union_scan_kernel<<<1, 1024, 0, s>>>(cnt, n, off);
    KW_TRY(cudaGetLastError());
    int m = 0;
    KW_TRY(cudaMemcpyAsync(&m, off + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    KW_TRY(cudaStreamSynchronize(s));
    if (m == 0) {
        out->ei.clear();
        out->ej.clear();
        out->w.clear();
        out->d2.clear();
        out->phi = phi_auto ? 0.0 : phi;
        cleanup();
        return cudaSuccess;
    }
    KW_TRY(cudaMalloc(&ei, sizeof(int) * (size_t)m));
    KW_TRY(cudaMalloc(&ej, sizeof(int) * (size_t)m));
    KW_TRY(cudaMalloc(&d2, sizeof(double) * (size_t)m));
    KW_TRY(cudaMalloc(&w, sizeof(double) * (size_t)m));
    count_launches(1);
    union_emit_kernel<<<row_blocks, kWThreads, 0, s>>>(bits, off, D, n, W, ei, ej, d2);
    KW_TRY(cudaGetLastError());
    // order statistics of d2 for the median (one rank when m is odd, the two middle ones when even);
    // the first histogram pass also takes the minimum
    const int hb = std::min(kWMaxBlocks, std::max(1, (m + kWThreads - 1) / kWThreads));
    const int nsel = phi_auto ? ((m & 1) ? 1 : 2) : (normalize ? 1 : 0);
    for (int r = 0; r < nsel; ++r) {
        const long long kth = phi_auto ? (long long)(m / 2) - ((m & 1) ? 0 : 1) + r : 0;
        count_launches(1);
        scalars_init_kernel<<<1, 1, 0, s>>>(sc, kth);
        for (int shift = 56; shift >= 0; shift -= 8) {
            count_launches(2);
            select_hist_kernel<<<hb, kWThreads, 0, s>>>(d2, m, sc, shift, r == 0 && shift == 56);
            select_pick_kernel<<<1, 1, 0, s>>>(sc, shift, r);
        }
        KW_TRY(cudaGetLastError());
    }
    count_launches(2);
    phi_kernel<<<1, 1, 0, s>>>(sc, m, phi, phi_auto);
    weight_kernel<<<hb, kWThreads, 0, s>>>(d2, m, sc, normalize, w, part);
    if (normalize) {
        count_launches(2);
        weight_total_kernel<<<1, 1, 0, s>>>(part, hb, sc);
        weight_scale_kernel<<<(m + kWThreads - 1) / kWThreads, kWThreads, 0, s>>>(w, m, sc);
    }
    KW_TRY(cudaGetLastError());
    out->ei.resize(m);
    out->ej.resize(m);
    out->w.resize(m);
    out->d2.resize(m);
    double phi_dev = 0.0;
    KW_TRY(cudaMemcpyAsync(out->ei.data(), ei, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost, s));
    KW_TRY(cudaMemcpyAsync(out->ej.data(), ej, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost, s));
    KW_TRY(cudaMemcpyAsync(out->w.data(), w, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, s));
    KW_TRY(cudaMemcpyAsync(out->d2.data(), d2, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, s));
    KW_TRY(cudaMemcpyAsync(&phi_dev, &sc->phi, sizeof(double), cudaMemcpyDeviceToHost, s));
    KW_TRY(cudaStreamSynchronize(s));
#undef KW_TRY
    out->phi = phi_dev;
    cleanup();
    return cudaSuccess;
}

}  // namespace ccx
