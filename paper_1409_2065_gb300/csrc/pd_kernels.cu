// Kernels of the proximal distance (PD) MM iteration for convex clustering.
//
// The paper's MM step (Methods, "The Proximal Distance Algorithm", Eq. 5 and
// the U- and V-update displays after it; "Missing Data", Eq. 6-7) is, for the
// iterate (U_m, V_m):
//     (A, B) = P_C(U_m, V_m):  (I + L) A = U_m + D^T V_m,  B = D A
//     d_m    = sqrt(||U_m - A||^2 + ||V_m - B||^2 + eps)
//     U_m+1  = (d_m Y + rho A) / (d_m + rho),  Y = X on observed entries, U_m elsewhere
//     v_ij   = max(1 - mu w_ij d_m / (rho ||b_ij||), 0) b_ij   (0 when b_ij = 0)
// This file runs that map with three changes of representation that leave its
// fixed point unchanged:
//   * V is never stored.  Since V_m+1 = s (.) D A_m, only the per-edge scalar
//     t = 1 - s and the previous projection are kept; D^T V and V - B are
//     formed from differences of projection rows on the fly.
//   * The projection is one Jacobi sweep of the paper's block update
//     (a_i = (r_i + sum_{N_i} a_j) / (1 + |N_i|)), written as a correction
//     delta of the extrapolated previous projection, so every term is a small
//     difference that keeps full relative precision in FP32.  A itself is
//     accumulated in float-float (FP32 path) or double (FP64 path).
//   * The map is applied at a Nesterov-extrapolated point (U_y, V_y, A_start)
//     with restarts (when <a_start - A_m, A_m - A_m-1> > 0); the extrapolated
//     warm start of the sweep keeps the inexact projection stable.
// U is held as the offset E = U - A_prev (small), so for observed entries it
// is recomputed from X, A and the scalar alpha = d / (d + rho) and never
// stored; missing entries keep two offsets (Q = U_y - A, Em = U - A_prev).
//
// Per iteration the work is two launches:
//   pd_slice_kernel : each CTA owns column slices of all n rows; for every
//                     slice it stages A_m-1 and Delta_m-1 in shared memory,
//                     updates all nodes (node phase), then runs the edge
//                     phase on the new rows (per-edge ||b||^2, ||V_y - B||^2).
//                     Columns are independent in both phases, so nothing but
//                     per-edge and scalar partial sums leaves the CTA.
//   pd_reduce_kernel: sums the partials in a fixed order (deterministic, no
//                     float atomics), forms d_m, the fused decision
//                     mu w d >= rho ||b||, t_m+1, and (last block) updates
//                     the scalar state: alpha, restart/beta, convergence.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "ccx_internal.h"

namespace ccx {
namespace {

template <typename R, int C>
struct alignas(sizeof(R) * C) Vec {
    R v[C];
};

constexpr int C = kSliceCols;
constexpr uint32_t kSliceMask = (C >= 32) ? 0xFFFFFFFFu : ((1u << C) - 1u);   // mask bits of one slice

__device__ __forceinline__ void ff_add(float hi, float lo, float inc, float& ohi, float& olo) {
    // (hi, lo) + inc in float-float: two-sum of hi and inc, then renormalise.
    const float s = __fadd_rn(hi, inc);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(inc, bb));
    const float l = __fadd_rn(lo, err);
    const float h2 = __fadd_rn(s, l);
    olo = __fsub_rn(l, __fsub_rn(h2, s));
    ohi = h2;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum; result valid in thread 0.  `red` holds >= 32 doubles.
__device__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < nw; ++k) r += red[k];
    }
    return r;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

// ------------------------------------------------------------------ slice
// 16-byte asynchronous global->shared copy (cp.async.cg bypasses L1).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T>
__device__ __forceinline__ void copy_vec_async(T* dst, const T* src) {
    static_assert(sizeof(T) % 16 == 0, "vector rows are multiples of 16 bytes");
#pragma unroll
    for (int k = 0; k < (int)(sizeof(T) / 16); ++k)
        cp_async16(reinterpret_cast<char*>(dst) + 16 * k, reinterpret_cast<const char*>(src) + 16 * k);
}

// Shared-memory layout of the iteration kernel (all offsets multiples of 16 bytes):
//   per staging buffer b in {0, 1 (prefetch only)}:
//       A_hi[n], (A_lo[n] on the FP32 path), Delta_{m-1}[n], X[n], mask word[n] (padded)
//   Delta_m[n]
//   Gpart[nslots]                (partial correction sums of the node-sweep runs)
//   rowptr[n + 1], erow[n + 1], ps0[n + 1]
//   nbacc[le*T]                  (float: this CTA's sum of ||b_m||^2 over its slices)
//   csrT[la*T], ejT[le*T]        (uint16 neighbour indices of the two sweeps)
template <typename R>
struct SliceLayout {
    static constexpr bool FF = std::is_same<R, float>::value;
    static constexpr size_t row = sizeof(R) * C;             // bytes of one row slice
    __host__ __device__ static size_t mask_bytes(int n) { return ((size_t)n * 4 + 15) / 16 * 16; }
    // A_hi (+A_lo) + Delta_{m-1} + X, then the mask words
    static size_t buf(int n) { return (FF ? 4 : 3) * row * (size_t)n + mask_bytes(n); }
    // stream: the per-entry arrays (neighbour indices, per-edge accumulators) stay
    // in global memory, for problems whose edge set does not fit beside the rows
    static size_t bytes(int n, int la, int le, int nslots, bool pref, bool stream) {
        const size_t LA = (size_t)la * kSliceThreads, LE = (size_t)le * kSliceThreads;
        size_t b = (pref ? 2 : 1) * buf(n) + row * (size_t)n;
        b += row * (size_t)nslots;
        b += sizeof(int) * 3 * (size_t)(n + 1);
        b = (b + 15) / 16 * 16;
        if (!stream) {
            b += sizeof(float) * LE;
            b += sizeof(uint16_t) * (LA + LE);
        }
        return (b + 15) / 16 * 16;
    }
};

template <typename R, bool PREF, bool STREAM>
__global__ void __launch_bounds__(kSliceThreads, 1) pd_slice_kernel(IterParams<R> P) {
    constexpr bool FF = std::is_same<R, float>::value;
    using V = Vec<R, C>;
    using VF = Vec<float, C>;
    const PdState* st = P.st;
    if (st->done) return;

    constexpr int T = kSliceThreads;
    const int n = P.n, ld = P.ld, m = P.m, tid = threadIdx.x, G = gridDim.x;
    const int la = P.la, le = P.le, LA = la * T, LE = le * T;
    // this thread's runs of the node sweep (CSR positions) and of the edge sweep (edge ids)
    const int qA0 = tid * la, nA = max(0, min(la, 2 * m - qA0));
    const int eE0 = tid * le, nE = max(0, min(le, m - eE0));
    const uint2 thrA = P.thrA[tid];
    const int iE0 = P.thrE[tid];
    const int par = st->par;
    const R beta = (R)st->beta;
    const R onepb = (R)(1.0 + st->beta);
    const R alpha1 = (R)st->alpha1;
    const R alpha2 = (R)st->alpha2;
    const R* __restrict__ Ahi_in = P.Ahi[par];
    const float* __restrict__ Alo_in = P.Alo[par];
    R* __restrict__ Ahi_out = P.Ahi[par ^ 1];
    float* __restrict__ Alo_out = P.Alo[par ^ 1];
    const R* __restrict__ D1g = P.Dl[par];       // Delta_{m-1}
    R* __restrict__ D0g = P.Dl[par ^ 1];         // Delta_m (written)
    const Vec<R, 2>* __restrict__ tA = reinterpret_cast<const Vec<R, 2>*>(P.t[par]);  // (t_m, t_{m-1})
    const Vec<R, 2>* __restrict__ tE = tA + LA;
    const R* __restrict__ Xg = P.X;
    const uint32_t* __restrict__ maskg = P.mask;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sp = smem_raw;
    V* bAhi[2];
    VF* bAlo[2];
    V* bD1[2];
    V* bX[2];
    uint32_t* bM[2];
    for (int b = 0; b < (PREF ? 2 : 1); ++b) {
        bAhi[b] = reinterpret_cast<V*>(sp);
        sp += sizeof(V) * (size_t)n;
        bAlo[b] = reinterpret_cast<VF*>(sp);
        if (FF) sp += sizeof(VF) * (size_t)n;
        bD1[b] = reinterpret_cast<V*>(sp);
        sp += sizeof(V) * (size_t)n;
        bX[b] = reinterpret_cast<V*>(sp);
        sp += sizeof(V) * (size_t)n;
        bM[b] = reinterpret_cast<uint32_t*>(sp);
        sp += SliceLayout<R>::mask_bytes(n);
    }
    if (!PREF) {
        bAhi[1] = bAhi[0];
        bAlo[1] = bAlo[0];
        bD1[1] = bD1[0];
        bX[1] = bX[0];
        bM[1] = bM[0];
    }
    V* sD0 = reinterpret_cast<V*>(sp);
    sp += sizeof(V) * (size_t)n;
    V* sPart = reinterpret_cast<V*>(sp);
    sp += sizeof(V) * (size_t)P.nslots;
    int* sRow = reinterpret_cast<int*>(sp);
    int* sErow = sRow + n + 1;
    int* sPs0 = sErow + n + 1;
    sp += sizeof(int) * 3 * (size_t)(n + 1);
    sp = smem_raw + ((size_t)(sp - smem_raw) + 15) / 16 * 16;
    float* sNb;                 // per edge-sweep position: this CTA's sum of ||b_m||^2
    const uint16_t* sCsrT;      // neighbour indices of the two sweeps
    const uint16_t* sEjT;
    if constexpr (STREAM) {
        sNb = P.Pnb + (size_t)blockIdx.x * LE;   // this CTA's own row of the partials
        sCsrT = P.csrT;
        sEjT = P.ejT;
    } else {
        sNb = reinterpret_cast<float*>(sp);
        sp += sizeof(float) * (size_t)LE;
        uint16_t* ci = reinterpret_cast<uint16_t*>(sp);
        sCsrT = ci;
        sEjT = ci + LA;
    }
    __shared__ double red[32];

    auto stage = [&](int sl, int b) {
        const int c0 = sl * C;
        V* dA = b ? bAhi[1] : bAhi[0];
        VF* dL = b ? bAlo[1] : bAlo[0];
        V* dD = b ? bD1[1] : bD1[0];
        V* dX = b ? bX[1] : bX[0];
        uint32_t* dM = b ? bM[1] : bM[0];
        for (int i = tid; i < n; i += kSliceThreads) {
            const size_t off = (size_t)i * ld + c0;
            copy_vec_async(&dA[i], reinterpret_cast<const V*>(Ahi_in + off));
            copy_vec_async(&dD[i], reinterpret_cast<const V*>(D1g + off));
            copy_vec_async(&dX[i], reinterpret_cast<const V*>(Xg + off));
            if constexpr (FF) copy_vec_async(&dL[i], reinterpret_cast<const VF*>(Alo_in + off));
            if (maskg) cp_async4(&dM[i], maskg + (size_t)i * P.ldw + (c0 >> 5));
        }
        cp_async_commit();
    };

    int cur = 0;
    if (blockIdx.x < P.nslices) stage(blockIdx.x, 0);
    // launch-constant graph data
    for (int k = tid; k <= n; k += kSliceThreads) {
        sRow[k] = P.rowptr[k];
        sErow[k] = P.erow[k];
        sPs0[k] = P.ps0[k];
    }
    if constexpr (!STREAM) {
        uint16_t* ci = const_cast<uint16_t*>(sCsrT);
        for (int k = tid; k < LA; k += kSliceThreads) ci[k] = P.csrT[k];
        for (int k = tid; k < LE; k += kSliceThreads) ci[LA + k] = P.ejT[k];
    }
    // each thread clears the accumulator positions it owns (k * T + tid)
    for (int k = tid; k < LE; k += kSliceThreads) sNb[k] = 0.f;
    // scalar partial sums: per warp, in double, accumulated slice by slice in a fixed order
    __shared__ double sAcc[kSliceThreads / 32][kNumScalarPartials];
    for (int k = tid; k < (kSliceThreads / 32) * kNumScalarPartials; k += kSliceThreads) (&sAcc[0][0])[k] = 0.0;
    const int warp = tid >> 5, lane = tid & 31;
    auto flush = [&](float v, int slot) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sAcc[warp][slot] += (double)v;
    };

    for (int sl = blockIdx.x; sl < P.nslices; sl += G) {
        const int c0 = sl * C;
        if (!PREF && sl != (int)blockIdx.x) stage(sl, 0);
        cp_async_wait_all();
        __syncthreads();
        if (PREF && sl + G < P.nslices) stage(sl + G, cur ^ 1);
        const V* __restrict__ sAhi = cur ? bAhi[1] : bAhi[0];
        const VF* __restrict__ sAlo = cur ? bAlo[1] : bAlo[0];
        const V* __restrict__ sD1 = cur ? bD1[1] : bD1[0];
        const V* __restrict__ sX = cur ? bX[1] : bX[0];
        const uint32_t* __restrict__ sM = cur ? bM[1] : bM[0];

        // ---- node sweep: G_i = sum over neighbours of the extrapolated D^T V_y terms.
        //      Each thread walks its run of CSR entries in order; a partial sum is
        //      written whenever the run leaves a row (and at its end).
        if (nA > 0) {
            int i = (int)thrA.x, slot = (int)thrA.y, rend = sRow[i + 1];
            V a = sAhi[i];
            V d1 = sD1[i];
            VF al;
            if constexpr (FF) al = sAlo[i];
            R G_[C];
#pragma unroll
            for (int c = 0; c < C; ++c) G_[c] = (R)0;
            Vec<R, 2> tn0 = tA[tid], tn1;
            if (nA > 1) tn1 = tA[T + tid];
            // the neighbour rows of entry k + 1 are requested while entry k is summed
            int jn = sCsrT[tid];
#pragma unroll 2
            for (int k = 0; k < nA; ++k) {
                const Vec<R, 2> t2 = tn0;
                tn0 = tn1;
                if (k + 2 < nA) tn1 = tA[(k + 2) * T + tid];
                const int jc = jn;
                if (k + 1 < nA) jn = sCsrT[(k + 1) * T + tid];
                const V cbj = sAhi[jc], cdj = sD1[jc];
                VF clj;
                if constexpr (FF) clj = sAlo[jc];
                if (qA0 + k == rend) {
                    V gp;
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        gp.v[c] = G_[c];
                        G_[c] = (R)0;
                    }
                    sPart[slot++] = gp;
                    do {
                        ++i;
                        rend = sRow[i + 1];
                    } while (rend <= qA0 + k);
                    a = sAhi[i];
                    d1 = sD1[i];
                    if constexpr (FF) al = sAlo[i];
                }
                // (1+beta) t_m b1 - beta t_{m-1} b2 with b2 = b1 - (d1_i - d1_j)
                const R cb = beta * t2.v[1];
                const R cd = onepb * t2.v[0] - cb;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    R b1 = a.v[c] - cbj.v[c];
                    if constexpr (FF) b1 += al.v[c] - clj.v[c];
                    G_[c] = fma(cd, b1, G_[c]);
                    G_[c] = fma(cb, d1.v[c] - cdj.v[c], G_[c]);
                }
            }
            V gp;
#pragma unroll
            for (int c = 0; c < C; ++c) gp.v[c] = G_[c];
            sPart[slot] = gp;
        }
        __syncthreads();

        // ---- node phase B: one preconditioned correction of the projection per (i, slice)
        float f_ua = 0.f, f_rs = 0.f, f_st = 0.f, f_na = 0.f, f_nz = 0.f, f_dl = 0.f;
        // missing entries of this thread's first two nodes: issue their loads together
        V qv0, qv1, ev0, ev1;
        if (maskg) {
            const int i0 = tid, i1 = tid + kSliceThreads;
            if (i0 < n && ((sM[i0] >> (c0 & 31)) & kSliceMask) != kSliceMask) {
                qv0 = *reinterpret_cast<const V*>(P.Q + (size_t)i0 * ld + c0);
                ev0 = *reinterpret_cast<const V*>(P.Em + (size_t)i0 * ld + c0);
            }
            if (i1 < n && ((sM[i1] >> (c0 & 31)) & kSliceMask) != kSliceMask) {
                qv1 = *reinterpret_cast<const V*>(P.Q + (size_t)i1 * ld + c0);
                ev1 = *reinterpret_cast<const V*>(P.Em + (size_t)i1 * ld + c0);
            }
        }
        for (int i = tid, u = 0; i < n; i += kSliceThreads, ++u) {
            const size_t off = (size_t)i * ld + c0;
            const V x = sX[i];
            const uint32_t obs = maskg ? (sM[i] >> (c0 & 31)) & kSliceMask : kSliceMask;
            V qv, ev;
            if (obs != kSliceMask) {
                if (u == 0) {
                    qv = qv0;
                    ev = ev0;
                } else if (u == 1) {
                    qv = qv1;
                    ev = ev1;
                } else {
                    qv = *reinterpret_cast<const V*>(P.Q + off);
                    ev = *reinterpret_cast<const V*>(P.Em + off);
                }
            }
            const V a = sAhi[i];
            const V d1 = sD1[i];
            VF al;
            if constexpr (FF) al = sAlo[i];
            R G_[C];
#pragma unroll
            for (int c = 0; c < C; ++c) G_[c] = (R)0;
            for (int k = sPs0[i]; k < sPs0[i + 1]; ++k) {     // fixed order: deterministic
                const V gp = sPart[k];
#pragma unroll
                for (int c = 0; c < C; ++c) G_[c] += gp.v[c];
            }
            // preconditioner P = I + 2 Deg >= I + L: the sweep's iteration matrix
            // has eigenvalues in [0, 1), which the extrapolation needs
            const R inv = (R)1 / (R)(1 + 2 * (sRow[i + 1] - sRow[i]));
            V dm;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                R lo = (R)0;
                if constexpr (FF) lo = al.v[c];
                R Em, Em1;
                if (obs & (1u << c)) {
                    const R xm = (x.v[c] - a.v[c]) - lo;      // y - a_{m-1}
                    Em = alpha1 * xm;                          // U_m - A_{m-1}
                    Em1 = alpha2 * (xm + d1.v[c]);             // U_{m-1} - A_{m-2}
                } else {
                    Em = alpha1 * qv.v[c];
                    Em1 = ev.v[c];
                }
                const R ue = onepb * Em - beta * Em1;          // U_y - A_start
                const R delta = (ue - G_[c]) * inv;            // A_m - A_start
                const R inc = beta * d1.v[c] + delta;          // A_m - A_{m-1}
                dm.v[c] = inc;
                if (!(obs & (1u << c))) {
                    P.Q[off + c] = ue - delta;                 // U_y - A_m
                    P.Em[off + c] = Em;
                }
                const float nz = (float)((fabs(ue) + fabs(G_[c])) * inv);
                f_nz += nz * nz;
                f_dl += (float)(delta * delta);
                const float r_ua = (float)(ue - delta);
                f_ua += r_ua * r_ua;
                f_rs -= (float)(delta * inc);
                f_st += (float)(inc * inc);
            }
            if constexpr (FF) {
                V ohi;
                VF olo;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    float h, l;
                    ff_add(a.v[c], al.v[c], dm.v[c], h, l);
                    ohi.v[c] = h;
                    olo.v[c] = l;
                    f_na += h * h;
                }
                *reinterpret_cast<V*>(Ahi_out + off) = ohi;
                *reinterpret_cast<VF*>(Alo_out + off) = olo;
            } else {
                V ohi;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    ohi.v[c] = a.v[c] + dm.v[c];
                    f_na += (float)(ohi.v[c] * ohi.v[c]);
                }
                *reinterpret_cast<V*>(Ahi_out + off) = ohi;
            }
            *reinterpret_cast<V*>(D0g + off) = dm;
            sD0[i] = dm;
        }
        __syncthreads();

        flush(f_ua, kPsUA);
        flush(f_rs, kPsRestart);
        flush(f_st, kPsStep);
        flush(f_na, kPsNormA);
        flush(f_nz, kPsNoise);
        flush(f_dl, kPsDelta);

        // ---- edge sweep: b_m = b_{m-1} + (Delta_m,i - Delta_m,j); ||b_m||^2 per edge
        //      and ||V_y - B_m||^2.  Each thread walks its run of edges (sorted by
        //      (i, j)), reloading the smaller endpoint's rows when i changes.
        float f_vb = 0.f;
        if (nE > 0) {
            int i = iE0, rend = sErow[i + 1];
            V a = sAhi[i];
            V d1 = sD1[i];
            V d0 = sD0[i];
            VF al;
            if constexpr (FF) al = sAlo[i];
            Vec<R, 2> tn0 = tE[tid], tn1;
            if (nE > 1) tn1 = tE[T + tid];
            int jn = sEjT[tid];
#pragma unroll 2
            for (int k = 0; k < nE; ++k) {
                const Vec<R, 2> t2 = tn0;
                tn0 = tn1;
                if (k + 2 < nE) tn1 = tE[(k + 2) * T + tid];
                const int jc = jn;
                if (k + 1 < nE) jn = sEjT[(k + 1) * T + tid];
                const V cbj = sAhi[jc], cd1j = sD1[jc], cd0j = sD0[jc];
                VF clj;
                if constexpr (FF) clj = sAlo[jc];
                if (eE0 + k == rend) {
                    do {
                        ++i;
                        rend = sErow[i + 1];
                    } while (rend <= eE0 + k);
                    a = sAhi[i];
                    d1 = sD1[i];
                    d0 = sD0[i];
                    if constexpr (FF) al = sAlo[i];
                }
                // V_y - B_m = -(dmv - beta d1v) - ((1+beta) t_m b1 - beta t_{m-1} b2),
                // b2 = b1 - d1v:  = -dmv + (beta - tb) d1v - (ta - tb) b1
                const R tb = beta * t2.v[1];
                const R q1 = beta - tb;
                const R q2 = tb - onepb * t2.v[0];
                R sb = (R)0, sv = (R)0;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    R b1 = a.v[c] - cbj.v[c];
                    if constexpr (FF) b1 += al.v[c] - clj.v[c];
                    const R d1v = d1.v[c] - cd1j.v[c];
                    const R dmv = d0.v[c] - cd0j.v[c];
                    const R b = b1 + dmv;                   // b_m
                    const R vmb = fma(q2, b1, fma(q1, d1v, -dmv));
                    sb = fma(b, b, sb);
                    sv = fma(vmb, vmb, sv);
                }
                sNb[k * T + tid] += (float)sb;   // position owned by this thread
                f_vb += (float)sv;
            }
        }
        flush(f_vb, kPsVB);
        __syncthreads();
        cur ^= (PREF ? 1 : 0);
    }

    // ---- partials of this CTA
    if constexpr (!STREAM)
        for (int k = tid; k < LE; k += kSliceThreads) P.Pnb[(size_t)blockIdx.x * LE + k] = sNb[k];
    double* ps = P.Ps + (size_t)blockIdx.x * kNumScalarPartials;
    if (tid < kNumScalarPartials) {
        double r = 0.0;
        for (int w = 0; w < kSliceThreads / 32; ++w) r += sAcc[w][tid];
        ps[tid] = r;
    }
}

// ------------------------------------------------------------------ reduce
// Block = 32 edges x 8 CTA groups.  Each edge's partials are summed in a fixed
// order (CTA group, then group index), so results do not depend on timing.
constexpr int kRedEdges = 32;
constexpr int kRedGroups = kReduceThreads / kRedEdges;

// Sum of the d_m pieces ||U_y - A_m||^2 + ||V_y - B_m||^2 over G partial rows
// of stride `stride` (lane-strided, then a shuffle tree; valid in lane 0).  The
// reduce kernel and the shard-partials kernel both use it, so one shard's
// total reproduces the unsharded sum exactly.
__device__ __forceinline__ double dm_sum(const double* ps, int G, long long stride, int lane) {
    double acc = 0.0;
    for (int g = lane; g < G; g += 32) acc += ps[(size_t)g * stride + kPsUA] + ps[(size_t)g * stride + kPsVB];
    return warp_sum(acc);
}

// Per edge-sweep position: the 8-group strided sum of the per-CTA ||b||^2
// partials (group q takes CTAs q, q + 8, ...), then the groups in order.
// The loads are issued four at a time ahead of their (in-order) additions, so a
// thread waits for one L2 round trip per four partials instead of per partial.
__device__ __forceinline__ double nb2_group_sum(const float* Pnb, int G, int LE, int pos, int grp) {
    double s = 0.0;
    int g = grp;
    for (; g + 3 * kRedGroups < G; g += 4 * kRedGroups) {
        const float v0 = Pnb[(size_t)g * LE + pos];
        const float v1 = Pnb[(size_t)(g + kRedGroups) * LE + pos];
        const float v2 = Pnb[(size_t)(g + 2 * kRedGroups) * LE + pos];
        const float v3 = Pnb[(size_t)(g + 3 * kRedGroups) * LE + pos];
        s += (double)v0;
        s += (double)v1;
        s += (double)v2;
        s += (double)v3;
    }
    for (; g < G; g += kRedGroups) s += (double)Pnb[(size_t)g * LE + pos];
    return s;
}

template <typename R>
__device__ void last_block_update(PdState* st, const double (*redv)[7], const unsigned long long* hsh,
                                  int nthreads, double d, double rho);

// This thread's share of ||a_i - a_j||^2 in double over the p columns of two rows
// of A (hi + lo on the FP32 path), rows starting at offsets oi and oj (multiples
// of 32 elements): groups of four columns, two groups in flight per step so that
// a thread waits for one L2 round trip per eight columns; the last p mod 4
// columns go to the first threads.  The order of the additions is fixed.
template <typename R>
__device__ __forceinline__ double row_diff_sq(const R* __restrict__ hi, const float* __restrict__ lo, size_t oi,
                                              size_t oj, int p, int tid) {
    constexpr bool FF = std::is_same<R, float>::value;
    using V4 = Vec<R, 4>;
    using F4 = Vec<float, 4>;
    constexpr int T = kReduceThreads;
    const int ng = p / 4;
    double acc0 = 0.0, acc1 = 0.0;
    auto group = [&](int g, double& acc) {
        const V4 hi4 = *reinterpret_cast<const V4*>(hi + oi + 4 * (size_t)g);
        const V4 hj4 = *reinterpret_cast<const V4*>(hi + oj + 4 * (size_t)g);
        F4 li4, lj4;
        if constexpr (FF) {
            li4 = *reinterpret_cast<const F4*>(lo + oi + 4 * (size_t)g);
            lj4 = *reinterpret_cast<const F4*>(lo + oj + 4 * (size_t)g);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double ai = (double)hi4.v[c], aj = (double)hj4.v[c];
            if constexpr (FF) {
                ai += (double)li4.v[c];
                aj += (double)lj4.v[c];
            }
            const double dd = ai - aj;
            acc = fma(dd, dd, acc);
        }
    };
    int g = tid;
    for (; g + T < ng; g += 2 * T) {
        group(g, acc0);
        group(g + T, acc1);
    }
    if (g < ng) group(g, acc0);
    const int c = 4 * ng + tid;
    if (c < p) {
        double ai = (double)hi[oi + c], aj = (double)hi[oj + c];
        if constexpr (FF) {
            ai += (double)lo[oi + c];
            aj += (double)lo[oj + c];
        }
        const double dd = ai - aj;
        acc0 = fma(dd, dd, acc0);
    }
    return acc0 + acc1;
}

template <typename R>
__global__ void __launch_bounds__(kReduceThreads) pd_reduce_kernel(IterParams<R> P) {
    constexpr bool FF = std::is_same<R, float>::value;
    PdState* st = P.st;
    if (st->done) return;
    __shared__ double s_d;
    __shared__ double part[kRedGroups][kRedEdges];
    __shared__ double s_nb[kRedEdges];
    __shared__ unsigned s_near;
    __shared__ bool s_last;
    __shared__ double red[32];
    const int G = P.G, tid = threadIdx.x;
    const int LA = P.la * kSliceThreads, LE = P.le * kSliceThreads;
    const double* ext = P.ext_part;
    if (tid < 32) {
        // d_m (Eq. 5): per-CTA partials (or the shards' totals, in shard order)
        const double acc = ext ? dm_sum(ext + LE, P.n_ext, P.ext_len, tid) : dm_sum(P.Ps, G, kNumScalarPartials, tid);
        if (tid == 0) s_d = sqrt(acc + st->eps);
    }
    // one lane per edge-sweep position pos = k*T + t, the k-th edge of run t
    const int lane = tid % kRedEdges, grp = tid / kRedEdges;
    const int pos = blockIdx.x * kRedEdges + lane;
    const int e = pos < LE ? P.eid[pos] : -1;
    // this edge's weight, previous t and node-sweep positions, requested before the
    // partial sums so that their round trip to L2 overlaps with those loads
    R told = (R)0;
    int2 qp = make_int2(0, 0);
    double we = 0.0;
    if (grp == 0 && e >= 0) {
        we = P.w[e];
        told = P.t[st->par][2 * (size_t)LA + 2 * (size_t)pos];
        qp = P.posA[pos];
    }
    double s = 0.0;
    if (e >= 0) {
        if (ext) {
            for (int q = grp; q < P.n_ext; q += kRedGroups) s += ext[(size_t)q * P.ext_len + pos];
        } else {
            s = nb2_group_sum(P.Pnb, G, LE, pos, grp);
        }
    }
    part[grp][lane] = s;
    __syncthreads();
    const double d = s_d;
    const double gamma = st->gamma, rho = st->rho;
    double lhs = 0.0;
    bool near = false;
    if (grp == 0) {
        double nb = 0.0;
        if (e >= 0) {
            double tot = 0.0;
            for (int g = 0; g < kRedGroups; ++g) tot += part[g][lane];
            nb = sqrt(tot);
            lhs = gamma * we * d;
            const double rhs = rho * nb;
            // the prox's zero test mu w d >= rho ||b|| within the rounding of the
            // float partial sums: decide it from ||b|| recomputed in double
            near = P.delta_fuse > 0.0 && rhs > 0.0 && fabs(lhs - rhs) <= P.delta_fuse * rhs;
        }
        s_nb[lane] = nb;
        const unsigned nm = __ballot_sync(0xffffffffu, near);
        if (lane == 0) s_near = nm;
    }
    __syncthreads();
    // FP64 recompute of ||a_i - a_j|| from the rows of A_m (written by this
    // iteration's slice kernel into the slots the next iteration reads), the
    // whole block on one edge at a time in lane order: fixed-order sums
    unsigned nm = s_near;
    if (nm) {
        const int po = st->par ^ 1;
        const R* __restrict__ hi = P.Ahi[po];
        const float* __restrict__ lo = P.Alo[po];
        while (nm) {
            const int l = __ffs(nm) - 1;
            nm &= nm - 1;
            const int ee = P.eid[blockIdx.x * kRedEdges + l];
            const size_t oi = (size_t)P.ei[ee] * P.ld, oj = (size_t)P.ej[ee] * P.ld;
            const double tot = block_sum(row_diff_sq<R>(hi, lo, oi, oj, P.p, tid), red);
            if (tid == 0) s_nb[l] = sqrt(tot);
            __syncthreads();
        }
    }
    if (grp == 0) {
        R* tAout = P.t[st->par ^ 1];          // (t_{m+1}, t_m) replaces (t_m, t_{m-1})
        R* tEout = tAout + 2 * (size_t)LA;
        bool fz = false;
        unsigned long long h = 0ULL;
        if (e >= 0) {
            const double nb = s_nb[lane];
            const double rhs = rho * nb;
            fz = lhs >= rhs;                 // the prox returns exactly zero
            const R tnew = fz ? (R)1 : (R)(lhs / rhs);
            tEout[2 * pos] = tnew;
            tEout[2 * pos + 1] = told;
            tAout[2 * qp.x] = tnew;                // qp: the edge's two node-sweep positions
            tAout[2 * qp.x + 1] = told;
            tAout[2 * qp.y] = tnew;
            tAout[2 * qp.y + 1] = told;
            P.nb[e] = nb;
            P.fused[e] = fz ? 1 : 0;
            // the stability test of the stopping rule follows only the clearly
            // fused edges: an edge on the threshold may flip at rounding level
            // for ever without the iterate changing
            if (lhs >= rhs * (1.0 + kFuseMargin)) h = mix64((unsigned long long)e + 1ULL);
        }
        const unsigned ballot = __ballot_sync(0xffffffffu, fz);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
        if (lane == 0) {
            P.Rf[3 * blockIdx.x] = (unsigned long long)__popc(ballot);
            P.Rf[3 * blockIdx.x + 1] = h;
            P.Rf[3 * blockIdx.x + 2] = (unsigned long long)__popc(s_near);
            __threadfence();
            const unsigned int ticket = atomicAdd(&st->counter, 1u);
            s_last = (ticket == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // ---- last block: scalar state update (block-parallel fixed-order sums, then thread 0)
    unsigned long long nf_l = 0ULL, hash_l = 0ULL, nr_l = 0ULL;
    for (int b = tid; b < (int)gridDim.x; b += blockDim.x) {
        nf_l += P.Rf[3 * b];
        hash_l += P.Rf[3 * b + 1];
        nr_l += P.Rf[3 * b + 2];
    }
    double q_rs = 0.0, q_st = 0.0, q_na = 0.0, q_nz = 0.0, q_dl = 0.0;
    {
        const double* base = ext ? ext + LE : P.Ps;
        const long long stride = ext ? P.ext_len : kNumScalarPartials;
        const int rows = ext ? P.n_ext : G;
        for (int g = tid; g < rows; g += blockDim.x) {
            const double* ps = base + (size_t)g * stride;
            q_rs += ps[kPsRestart];
            q_st += ps[kPsStep];
            q_na += ps[kPsNormA];
            q_nz += ps[kPsNoise];
            q_dl += ps[kPsDelta];
        }
    }
    // seven block sums in one pass, each in the order of block_sum: a shuffle
    // tree per warp, then the warps in order
    constexpr int kNv = 7;
    double v[kNv] = {q_rs, q_st, q_na, q_nz, q_dl, (double)nf_l, (double)nr_l};
    __shared__ double redv[kReduceThreads / 32][kNv];
    __shared__ unsigned long long hsh[kReduceThreads];
#pragma unroll
    for (int k = 0; k < kNv; ++k) v[k] = warp_sum(v[k]);
    if ((tid & 31) == 0)
#pragma unroll
        for (int k = 0; k < kNv; ++k) redv[tid >> 5][k] = v[k];
    hsh[tid] = hash_l;
    // the scalar state, copied to shared memory for thread 0's serial update: one
    // coalesced read and write instead of a dependent global round trip per field
    static_assert(sizeof(PdState) % 8 == 0, "PdState is copied as 8-byte words");
    constexpr int kStWords = (int)(sizeof(PdState) / 8);
    __shared__ unsigned long long s_state[kStWords];
    for (int k = tid; k < kStWords; k += blockDim.x)
        s_state[k] = reinterpret_cast<const unsigned long long*>(P.st)[k];
    __syncthreads();
    if (tid == 0) last_block_update<R>(reinterpret_cast<PdState*>(s_state), redv, hsh, blockDim.x, d, rho);
    __syncthreads();
    for (int k = tid; k < kStWords; k += blockDim.x) reinterpret_cast<unsigned long long*>(P.st)[k] = s_state[k];
}

// Thread 0 of the reduction's last block: the iteration's scalar state update
// (d_m, alpha, momentum, the fused-set stability and the stopping rule) on the
// state `st` held in shared memory.
template <typename R>
__device__ void last_block_update(PdState* st, const double (*redv)[7], const unsigned long long* hsh,
                                  int nthreads, double d, double rho) {
    constexpr int kNv = 7;
    double tv[kNv];
#pragma unroll
    for (int k = 0; k < kNv; ++k) {
        tv[k] = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) tv[k] += redv[w][k];
    }
    const double rs = tv[0], stp = tv[1], na = tv[2], nzs = tv[3], dls = tv[4];
    const unsigned long long nf = (unsigned long long)tv[5];
    const unsigned long long nrec = (unsigned long long)tv[6];
    unsigned long long hash = 0ULL;
    for (int k = 0; k < nthreads; ++k) hash += hsh[k];
    const double unit = sizeof(R) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
    const double noise = unit * sqrt(nzs);
    st->iter += 1;
    st->n_recomputed = (int)nrec;
    st->recompute_total += (long long)nrec;
    st->d_last = d;
    st->alpha2 = st->alpha1;
    st->alpha1 = d / (d + rho);
    if (st->aa_on) {
        // Anderson mixing phase (aa_kernels.cu): the plain map, no momentum
        st->k_mom = 0;
        st->beta = 0.0;
    } else if (st->accelerate) {
        // adaptive restart (O'Donoghue-Candes gradient test) on the projection:
        // drop the momentum when <a_start - A_m, A_m - A_{m-1}> > 0
        if (rs > 0.0) st->k_mom = 0;
        else st->k_mom += 1;
        const int k = st->k_mom;
        st->beta = k >= 1 ? (double)(k - 1) / (double)(k + 2) : 0.0;
    } else {
        st->beta = 0.0;
    }
    if (hash == st->fused_hash) st->fused_stable += 1;
    else st->fused_stable = 0;
    st->n_fused = (int)nf;
    st->fused_hash = hash;
    const double step = sqrt(stp);
    const double an = sqrt(na);
    st->a_norm = an;
    const double dres = sqrt(dls);
    if (step > st->blk_max) st->blk_max = step;
    if (noise > st->noise_max) st->noise_max = noise;
    if (dres > st->dmax) st->dmax = dres;
    if (st->iter % kConvWindow == 0 && !st->aa_on) {
        // Error estimate.  The correction ||A_m - A_start|| is the map's residual
        // at the extrapolated point: ~ eta * error for the slowest mode (gap eta),
        // and unlike the step it does not jump when the momentum restarts.  The
        // extrapolated iteration shrinks the error by ~(1 - sqrt(eta)) per step,
        // so the residual's observed log-decay per iteration g over the last
        // kRateWindows windows gives eta ~ g^2 and error ~ residual / g^2.
        const double cur = st->dmax;
        // error scale ||A||, floored at the rounding level of the data (matters
        // only when the centroids are ~0, e.g. fully fused centred data)
        const double scale = fmax(an, st->scale_floor);
        double est = INFINITY;
        const bool full = st->ring_len == kRateWindows;
        if (cur == 0.0) {
            est = 0.0;
        } else if (full && cur < st->ring[0]) {
            const double g = log(st->ring[0] / cur) / (double)(kRateWindows * kConvWindow);
            est = cur / (g * g) / scale;
            if (cur <= 0.5 * st->ring[0]) st->g_last = g;
        }
        st->err_est = est;
        // plateau: the residual has stopped falling (rounding level of this
        // state); its error is the plateau residual over the last measured rate
        const bool stalled = full && cur > 0.5 * st->ring[0];
        st->stall_hits = stalled ? st->stall_hits + 1 : 0;
        double est_plateau = INFINITY;
        if (st->g_last > 0.0) est_plateau = cur / (st->g_last * st->g_last) / scale;
        if (est <= st->tol && st->fused_stable >= kConvWindow) st->hits += 1;
        else st->hits = 0;
        // steps at the rounding level of their own inputs: no further progress
        if (st->tol >= 0.0 && st->blk_max <= kNoiseFactor * st->noise_max && st->fused_stable >= kConvWindow)
            st->floor_hits += 1;
        else st->floor_hits = 0;
        if (st->hits >= 2) {
            st->done = 1;
            st->converged = 1;
        } else if (st->floor_hits >= kNoiseWindows) {
            st->done = 1;
            st->converged = 2;
            st->err_est = st->blk_max * kStallSteps / scale;
        } else if (st->stall_hits >= kStallWindows && st->fused_stable >= kStallWindows * kConvWindow &&
                   est_plateau <= kStallTolFactor * st->tol && cur <= unit * sqrt(unit) * scale) {
            // (a slowly converging mode also looks flat over a few windows; its
            // residual is far above u^1.5 of the solution's scale)
            st->done = 1;
            st->converged = 2;
            st->err_est = est_plateau;
        }
        for (int q = 0; q + 1 < kRateWindows; ++q) st->ring[q] = st->ring[q + 1];
        st->ring[kRateWindows - 1] = cur;
        if (st->ring_len < kRateWindows) st->ring_len += 1;
        st->blk_max = 0.0;
        st->noise_max = 0.0;
        st->dmax = 0.0;
    }
    if (!st->done && st->iter >= st->max_iter) {
        st->done = 1;
        st->converged = 0;
    }
    st->par ^= 1;
    st->counter = 0u;
}


// One shard's partials of the iteration: per edge-sweep position the ||b||^2
// partials of its G CTAs summed as pd_reduce_kernel sums them (8 strided
// groups, then the groups in order), and the scalar partials summed as that
// kernel's d_m and last block sum them.  With one shard the reduction over
// these totals is therefore bit-identical to the unsharded one.
template <typename R>
__global__ void __launch_bounds__(kReduceThreads) pd_shard_partials_kernel(IterParams<R> P, double* __restrict__ out) {
    if (P.st->done) return;
    const int G = P.G, tid = threadIdx.x, LE = P.le * kSliceThreads;
    __shared__ double part[kRedGroups][kRedEdges];
    __shared__ double red[32];
    const int lane = tid % kRedEdges, grp = tid / kRedEdges;
    const int pos = blockIdx.x * kRedEdges + lane;
    if (blockIdx.x * kRedEdges < LE) {
        part[grp][lane] = pos < LE ? nb2_group_sum(P.Pnb, G, LE, pos, grp) : 0.0;
        __syncthreads();
        if (grp == 0 && pos < LE) {
            double tot = 0.0;
            for (int g = 0; g < kRedGroups; ++g) tot += part[g][lane];
            out[pos] = tot;
        }
        return;
    }
    // the extra last block: scalar partials
    if (tid < 32) {
        const double acc = dm_sum(P.Ps, G, kNumScalarPartials, tid);
        if (tid == 0) {
            out[LE + kPsUA] = acc;   // the two d_m pieces travel as one sum
            out[LE + kPsVB] = 0.0;
        }
    }
    const int slots[5] = {kPsRestart, kPsStep, kPsNormA, kPsNoise, kPsDelta};
    for (int k = 0; k < 5; ++k) {
        double q = 0.0;
        for (int g = tid; g < G; g += blockDim.x) q += P.Ps[(size_t)g * kNumScalarPartials + slots[k]];
        const double t = block_sum(q, red);
        if (tid == 0) out[LE + slots[k]] = t;
    }
    if (tid == 0) out[LE + 7] = 0.0;
}

// ------------------------------------------------------------------ init / begin / finalize
template <typename R>
__global__ void pd_init_kernel(IterParams<R> P, const R* Y0, size_t total) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        P.Ahi[0][k] = Y0[k];
        P.Ahi[1][k] = Y0[k];
        P.Dl[0][k] = (R)0;
        P.Dl[1][k] = (R)0;
        if constexpr (std::is_same<R, float>::value) {
            P.Alo[0][k] = 0.f;
            P.Alo[1][k] = 0.f;
        }
        if (P.Q) {
            P.Q[k] = (R)0;
            P.Em[k] = (R)0;
        }
    }
    const size_t npairs = ((size_t)P.la + P.le) * kSliceThreads;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < 2 * npairs; q += (size_t)gridDim.x * blockDim.x) {
        P.t[0][q] = (R)1;   // t = 1 - s with s = 0: V_0 = 0 (and V_{-1} = 0)
        P.t[1][q] = (R)1;
    }
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)P.m; e += (size_t)gridDim.x * blockDim.x) {
        P.nb[e] = 0.0;
        P.fused[e] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        PdState* st = P.st;
        st->alpha1 = 0.0;
        st->alpha2 = 0.0;
        st->beta = 0.0;
        st->k_mom = 0;
        st->par = 0;
        st->iter = 0;
        st->done = 1;
        st->converged = 0;
        st->n_fused = -1;
        st->fused_hash = 0ULL;
        st->fused_stable = 0;
        st->counter = 0u;
        st->d_last = 0.0;
        st->n_recomputed = 0;
        st->recompute_total = 0;
        st->aa_on = 0;
        st->aa_total = 0;
    }
}

__global__ void pd_begin_gamma_kernel(PdState* st, double gamma, double rho, double eps, double tol, int max_iter,
                                      int accelerate, double scale_floor, int aa_m) {
    st->scale_floor = scale_floor;
    st->gamma = gamma;
    st->rho = rho;
    st->eps = eps;
    st->tol = tol;
    st->max_iter = max_iter;
    st->accelerate = accelerate;
    st->iter = 0;
    st->done = 0;
    st->converged = 0;
    st->k_mom = 0;
    st->beta = 0.0;
    st->hits = 0;
    st->blk_max = 0.0;
    st->err_est = INFINITY;
    st->fused_stable = 0;
    st->noise_max = 0.0;
    st->ring_len = 0;
    st->floor_hits = 0;
    st->stall_hits = 0;
    st->g_last = 0.0;
    for (int q = 0; q < kRateWindows; ++q) st->ring[q] = 0.0;
    st->dmax = 0.0;
    st->counter = 0u;
    st->n_recomputed = 0;
    st->recompute_total = 0;
    st->aa_m = aa_m;
    st->aa_on = aa_m > 0 ? 1 : 0;
    st->aa_len = 0;
    st->aa_head = 0;
    st->aa_iters = 0;
    st->aa_total = 0;
    st->aa_have_prev = 0;
    st->aa_counter = 0u;
    st->aa_ra_prev = 0.0;
    st->aa_sa = 0.0;
    for (int q = 0; q < 4; ++q) st->aa_win[q] = 0.0;
    for (int j = 0; j < kAaMax; ++j) st->aa_g[j] = 0.0;
}

template <typename R>
__global__ void pd_finalize_kernel(IterParams<R> P, float* U_out, int64_t ld_out, int p) {
    const PdState* st = P.st;
    const int par = st->par;
    const double alpha = st->alpha1;
    const size_t total = (size_t)P.n * p;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k / p), c = (int)(k % p);
        const size_t off = (size_t)i * P.ld + c;
        const R hi = P.Ahi[par][off];
        R lo = (R)0;
        if constexpr (std::is_same<R, float>::value) lo = P.Alo[par][off];
        bool obs = true;
        if (P.mask) obs = (P.mask[(size_t)i * P.ldw + (c >> 5)] >> (c & 31)) & 1u;
        const R E = obs ? (R)alpha * ((P.X[off] - hi) - lo) : (R)alpha * P.Q[off];   // U_{m+1} - A_m
        U_out[(size_t)i * ld_out + c] = (float)(hi + (lo + E));
    }
}

template <typename R, bool PREF, bool STREAM>
cudaError_t launch_slice(const IterParams<R>& P, size_t smem, cudaStream_t s) {
    auto kern = pd_slice_kernel<R, PREF, STREAM>;
    // The shared-memory opt-in is a function attribute, not a stream
    // operation: it is raised once, to the device maximum, on the first
    // (uncaptured) launch so that launches inside graph capture need no call.
    static int raised = 0;
    if (!raised) {
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
        const int dyn = optin - (int)fa.sharedSizeBytes;   // static shared memory counts against the limit
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        raised = dyn;
    }
    if ((int)smem > raised) return cudaErrorInvalidValue;
    kern<<<P.G, kSliceThreads, smem, s>>>(P);
    return cudaGetLastError();
}

}  // namespace

size_t pd_slice_smem_bytes(int n, int la, int le, int nslots, bool fp64, bool prefetch, bool stream) {
    return fp64 ? SliceLayout<double>::bytes(n, la, le, nslots, prefetch, stream)
                : SliceLayout<float>::bytes(n, la, le, nslots, prefetch, stream);
}

constexpr size_t kPrefetchSmemMax = 160 * 1024;

int pd_reduce_blocks(int le) { return (le * kSliceThreads + kRedEdges - 1) / kRedEdges; }

// largest dynamic shared memory a block may use on this device (static part excluded)
static size_t slice_smem_limit() {
    static int lim = 0;
    if (!lim) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        lim = optin - 2048;
    }
    return (size_t)lim;
}

template <typename R>
cudaError_t launch_pd_slice_variant(const IterParams<R>& P, int variant, cudaStream_t s) {
    constexpr bool fp64 = std::is_same<R, double>::value;
    count_launches(1);
    // the double buffer is worth it only while at least ~96 KB of the SM's
    // 256 KB L1/shared array stays L1 for the per-edge weights and row loads
    // (variant 1 takes it whenever it fits; variant 2 never)
    const size_t lim = slice_smem_limit();
    if (P.stream_edges)
        return launch_slice<R, false, true>(P, pd_slice_smem_bytes(P.n, P.la, P.le, P.nslots, fp64, false, true), s);
    const size_t with_pref = pd_slice_smem_bytes(P.n, P.la, P.le, P.nslots, fp64, true, false);
    const size_t pref_cap = variant == 1 ? lim : kPrefetchSmemMax;
    if (variant != 2 && with_pref <= lim && with_pref <= pref_cap) return launch_slice<R, true, false>(P, with_pref, s);
    const size_t staged = pd_slice_smem_bytes(P.n, P.la, P.le, P.nslots, fp64, false, false);
    if (staged <= lim) return launch_slice<R, false, false>(P, staged, s);
    // edge set too large to stage beside the rows: indices and accumulators stay in global memory
    return launch_slice<R, false, true>(P, pd_slice_smem_bytes(P.n, P.la, P.le, P.nslots, fp64, false, true), s);
}

template <typename R>
cudaError_t launch_pd_slice(const IterParams<R>& P, cudaStream_t s) {
    return launch_pd_slice_variant<R>(P, 0, s);
}

template <typename R>
cudaError_t launch_pd_shard_partials(const IterParams<R>& P, double* out, cudaStream_t s) {
    count_launches(1);
    pd_shard_partials_kernel<R><<<pd_reduce_blocks(P.le) + 1, kReduceThreads, 0, s>>>(P, out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pd_reduce(const IterParams<R>& P, cudaStream_t s) {
    count_launches(1);
    pd_reduce_kernel<R><<<pd_reduce_blocks(P.le), kReduceThreads, 0, s>>>(P);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pd_iteration_variant(const IterParams<R>& P, int variant, cudaStream_t s) {
    cudaError_t e = launch_pd_slice_variant<R>(P, variant, s);
    if (e != cudaSuccess) return e;
    return launch_pd_reduce<R>(P, s);
}

template <typename R>
cudaError_t launch_pd_iteration(const IterParams<R>& P, cudaStream_t s) {
    return launch_pd_iteration_variant<R>(P, 0, s);
}

template <typename R>
cudaError_t launch_pd_init(const IterParams<R>& P, const R* Y0, cudaStream_t s) {
    const size_t total = (size_t)P.n * P.ld;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    count_launches(1);
    pd_init_kernel<R><<<blocks, 256, 0, s>>>(P, Y0, total);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pd_begin_gamma(const IterParams<R>& P, double gamma, double rho, double eps, double tol,
                                  int max_iter, int accelerate, double scale_floor, int aa_m, cudaStream_t s) {
    count_launches(1);
    pd_begin_gamma_kernel<<<1, 1, 0, s>>>(P.st, gamma, rho, eps, tol, max_iter, accelerate, scale_floor, aa_m);
    return cudaGetLastError();
}

// Predictor between gammas: A <- w0 A + w1 A_prev + w2 A_prev2 in the slot the
// next iteration reads, then A_prev2 <- A_prev and A_prev <- the old A.  The
// weights are the Lagrange extrapolation weights (w0 = 1, w1 = w2 = 0 only
// records A); a buffer whose weight is 0 is not read (it may not exist yet).
template <typename R>
__global__ void pd_extrapolate_kernel(IterParams<R> P, R* __restrict__ p1_hi, float* __restrict__ p1_lo,
                                      R* __restrict__ p2_hi, float* __restrict__ p2_lo, double w0, double w1,
                                      double w2, size_t total) {
    const int par = P.st->par;
    R* hi = P.Ahi[par];
    float* lo = P.Alo[par];
    const bool use1 = (w1 != 0.0), use2 = (w2 != 0.0);
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        if constexpr (std::is_same<R, float>::value) {
            const float h0 = hi[k], l0 = lo[k];
            const float h1 = p1_hi[k], l1 = p1_lo[k];
            if (use1 || use2) {
                double w = w0 * ((double)h0 + (double)l0);
                if (use1) w += w1 * ((double)h1 + (double)l1);
                if (use2) w += w2 * ((double)p2_hi[k] + (double)p2_lo[k]);
                const float h = (float)w;
                hi[k] = h;
                lo[k] = (float)(w - (double)h);
            }
            if (p2_hi) {
                p2_hi[k] = h1;
                p2_lo[k] = l1;
            }
            p1_hi[k] = h0;
            p1_lo[k] = l0;
        } else {
            const double v = hi[k], v1 = p1_hi[k];
            if (use1 || use2) {
                double w = w0 * v;
                if (use1) w += w1 * v1;
                if (use2) w += w2 * p2_hi[k];
                hi[k] = w;
            }
            if (p2_hi) p2_hi[k] = v1;
            p1_hi[k] = v;
        }
    }
}

template <typename R>
cudaError_t launch_pd_extrapolate(const IterParams<R>& P, R* p1_hi, float* p1_lo, R* p2_hi, float* p2_lo, double w0,
                                  double w1, double w2, cudaStream_t s) {
    const size_t total = (size_t)P.n * P.ld;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    count_launches(1);
    pd_extrapolate_kernel<R><<<blocks, 256, 0, s>>>(P, p1_hi, p1_lo, p2_hi, p2_lo, w0, w1, w2, total);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pd_finalize(const IterParams<R>& P, float* U_out, int64_t ld_out, int p, cudaStream_t s) {
    const size_t total = (size_t)P.n * p;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    count_launches(1);
    pd_finalize_kernel<R><<<blocks, 256, 0, s>>>(P, U_out, ld_out, p);
    return cudaGetLastError();
}

template cudaError_t launch_pd_iteration<float>(const IterParams<float>&, cudaStream_t);
template cudaError_t launch_pd_iteration_variant<float>(const IterParams<float>&, int, cudaStream_t);
template cudaError_t launch_pd_iteration_variant<double>(const IterParams<double>&, int, cudaStream_t);
template cudaError_t launch_pd_slice_variant<float>(const IterParams<float>&, int, cudaStream_t);
template cudaError_t launch_pd_slice_variant<double>(const IterParams<double>&, int, cudaStream_t);
template cudaError_t launch_pd_shard_partials<float>(const IterParams<float>&, double*, cudaStream_t);
template cudaError_t launch_pd_shard_partials<double>(const IterParams<double>&, double*, cudaStream_t);
template cudaError_t launch_pd_slice<float>(const IterParams<float>&, cudaStream_t);
template cudaError_t launch_pd_slice<double>(const IterParams<double>&, cudaStream_t);
template cudaError_t launch_pd_reduce<float>(const IterParams<float>&, cudaStream_t);
template cudaError_t launch_pd_reduce<double>(const IterParams<double>&, cudaStream_t);
template cudaError_t launch_pd_iteration<double>(const IterParams<double>&, cudaStream_t);
template cudaError_t launch_pd_init<float>(const IterParams<float>&, const float*, cudaStream_t);
template cudaError_t launch_pd_init<double>(const IterParams<double>&, const double*, cudaStream_t);
template cudaError_t launch_pd_begin_gamma<float>(const IterParams<float>&, double, double, double, double, int, int,
                                                  double, int, cudaStream_t);
template cudaError_t launch_pd_begin_gamma<double>(const IterParams<double>&, double, double, double, double, int, int,
                                                   double, int, cudaStream_t);
template cudaError_t launch_pd_extrapolate<float>(const IterParams<float>&, float*, float*, float*, float*, double,
                                                  double, double, cudaStream_t);
template cudaError_t launch_pd_extrapolate<double>(const IterParams<double>&, double*, float*, double*, float*, double,
                                                   double, double, cudaStream_t);
template cudaError_t launch_pd_finalize<float>(const IterParams<float>&, float*, int64_t, int, cudaStream_t);
template cudaError_t launch_pd_finalize<double>(const IterParams<double>&, float*, int64_t, int, cudaStream_t);

}  // namespace ccx
