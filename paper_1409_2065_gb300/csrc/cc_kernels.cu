// Clusters = connected components of the fused edges (an edge is fused when
// the paper's V update returns exactly zero for it), labelled 0, 1, ... by
// the rank of each component's smallest case index.
//
// One CTA, hook-to-smaller-root with path halving, repeated until no hook
// happens, then full compression and a rank scan.  Roots only ever point to
// smaller indices, so every component ends at its minimum index whatever the
// order in which threads hook: the labels are deterministic.  The loop is
// bounded by n + 1 rounds.  A round in which no thread hooks proves every fused
// edge joins one component; if even the last round hooked, the labels are not
// proven and the component count is written as -1, which the host reports as
// an error instead of returning the labels.
#include <cuda_runtime.h>

#include <cstdint>

#include "ccx_internal.h"

namespace ccx {
namespace {

constexpr int kCcThreads = 1024;

__device__ __forceinline__ int find_root(volatile int* parent, int x) {
    // path halving; parent[i] <= i always holds, so the walk ends at a root
    int px = parent[x];
    while (px != x) {
        const int gx = parent[px];
        parent[x] = gx;
        x = gx;
        px = parent[x];
    }
    return x;
}

__global__ void __launch_bounds__(kCcThreads) cc_kernel(int n, int m, const int* __restrict__ ei,
                                                        const int* __restrict__ ej, const uint8_t* __restrict__ fused,
                                                        int* parent, int* labels, int* n_clusters) {
    __shared__ int changed;
    __shared__ int wsum[32];
    for (int i = threadIdx.x; i < n; i += blockDim.x) parent[i] = i;
    __syncthreads();
    volatile int* vp = parent;
    __shared__ int settled;
    if (threadIdx.x == 0) settled = 0;
    for (int round = 0; round <= n; ++round) {
        if (threadIdx.x == 0) changed = 0;
        __syncthreads();
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            if (!fused[e]) continue;
            const int ra = find_root(vp, ei[e]);
            const int rb = find_root(vp, ej[e]);
            if (ra != rb) {
                const int lo = ra < rb ? ra : rb, hi = ra < rb ? rb : ra;
                atomicMin(&parent[hi], lo);
                changed = 1;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) parent[i] = find_root(vp, i);
        __syncthreads();
        if (!changed) {
            if (threadIdx.x == 0) settled = 1;
            break;
        }
        __syncthreads();
    }
    __syncthreads();
    // ranks of the roots: block scan of root flags in index order
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int flag = (i < n && parent[i] == i) ? 1 : 0;
        // inclusive warp scan
        int v = flag;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) wsum[wid] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                const int t = wsum[k];
                wsum[k] = acc;
                acc += t;
            }
        }
        __syncthreads();
        const int excl = carry + wsum[wid] + v - flag;
        if (i < n && flag) labels[i] = excl;   // rank of this root
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + flag;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int r = parent[i];
        if (r != i) labels[i] = labels[r];
    }
    if (threadIdx.x == 0) *n_clusters = settled ? carry : -1;
}

}  // namespace

cudaError_t launch_fused_labels(int n, int m, const int* ei, const int* ej, const uint8_t* fused, int* labels,
                                int* n_clusters, int* scratch, cudaStream_t s) {
    count_launches(1);
    cc_kernel<<<1, kCcThreads, 0, s>>>(n, m, ei, ej, fused, scratch, labels, n_clusters);
    return cudaGetLastError();
}

}  // namespace ccx
