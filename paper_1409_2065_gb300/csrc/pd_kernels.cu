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
template <typename R>
__global__ void __launch_bounds__(kSliceThreads, 1) pd_slice_kernel(IterParams<R> P) {
    constexpr bool FF = std::is_same<R, float>::value;
    using V = Vec<R, C>;
    using VF = Vec<float, C>;
    const PdState* st = P.st;
    if (st->done) return;

    const int n = P.n, ld = P.ld, m = P.m, tid = threadIdx.x;
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
    const R* __restrict__ tm = P.t[par];         // t_m
    const R* __restrict__ tm1 = P.t[par ^ 1];    // t_{m-1}
    const R* __restrict__ Xg = P.X;
    const uint32_t* __restrict__ maskg = P.mask;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* sAhi = reinterpret_cast<V*>(smem_raw);
    V* sD1 = sAhi + n;
    V* sOhi = sD1 + n;
    V* sD0 = sOhi + n;
    VF* sAlo = reinterpret_cast<VF*>(sD0 + n);
    VF* sOlo = sAlo + (FF ? n : 0);
    double* sNb = reinterpret_cast<double*>(sOlo + (FF ? n : 0));   // per-edge ||b||^2 over this CTA's slices
    __shared__ double red[32];
    for (int e = tid; e < m; e += kSliceThreads) sNb[e] = 0.0;
    double s_ua = 0.0, s_vb = 0.0, s_rs = 0.0, s_st = 0.0, s_na = 0.0, s_nz = 0.0, s_dl = 0.0;

    for (int sl = blockIdx.x; sl < P.nslices; sl += gridDim.x) {
        const int c0 = sl * C;
        // ---- stage A_{m-1} and Delta_{m-1} of this slice for all rows
        for (int i = tid; i < n; i += kSliceThreads) {
            const size_t off = (size_t)i * ld + c0;
            sAhi[i] = *reinterpret_cast<const V*>(Ahi_in + off);
            sD1[i] = *reinterpret_cast<const V*>(D1g + off);
            if constexpr (FF) sAlo[i] = *reinterpret_cast<const VF*>(Alo_in + off);
        }
        __syncthreads();

        // ---- node phase: one Jacobi correction per node (i, slice)
        for (int i = tid; i < n; i += kSliceThreads) {
            const size_t off = (size_t)i * ld + c0;
            const V a = sAhi[i];
            const V d1 = sD1[i];
            VF al;
            if constexpr (FF) al = sAlo[i];
            R G[C];
#pragma unroll
            for (int c = 0; c < C; ++c) G[c] = (R)0;
            const int r0 = P.rowptr[i], r1 = P.rowptr[i + 1];
            for (int q = r0; q < r1; ++q) {
                const int j = __ldg(P.col + q);
                const int e = __ldg(P.eid + q);
                const R ca = onepb * __ldg(tm + e);
                const R cb = beta * __ldg(tm1 + e);
                const V bj = sAhi[j];
                const V dj = sD1[j];
                VF lj;
                if constexpr (FF) lj = sAlo[j];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    R b1 = a.v[c] - bj.v[c];
                    if constexpr (FF) b1 += al.v[c] - lj.v[c];
                    const R b2 = b1 - (d1.v[c] - dj.v[c]);
                    G[c] += ca * b1 - cb * b2;
                }
            }
            const R inv = (R)1 / (R)(1 + (r1 - r0));
            const V x = *reinterpret_cast<const V*>(Xg + off);
            uint32_t obs = 0xFu;
            if (maskg) obs = (maskg[(size_t)i * P.ldw + (c0 >> 5)] >> (c0 & 31)) & 0xFu;
            V ohi, dm;
            VF olo;
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
                    Em = alpha1 * P.Q[off + c];
                    Em1 = P.Em[off + c];
                }
                const R ue = onepb * Em - beta * Em1;          // U_y - A_start
                const R delta = (ue - G[c]) * inv;             // A_m - A_start
                const R inc = beta * d1.v[c] + delta;          // A_m - A_{m-1}
                if constexpr (FF) {
                    float h, l;
                    ff_add(a.v[c], al.v[c], inc, h, l);
                    ohi.v[c] = h;
                    olo.v[c] = l;
                } else {
                    ohi.v[c] = a.v[c] + inc;
                }
                dm.v[c] = inc;
                if (!(obs & (1u << c))) {
                    P.Q[off + c] = ue - delta;                 // U_y - A_m
                    P.Em[off + c] = Em;
                }
                const double nz = ((double)fabs(ue) + (double)fabs(G[c])) * (double)inv;
                s_nz += nz * nz;
                s_dl += (double)delta * (double)delta;
                const double r_ua = (double)(ue - delta);
                s_ua += r_ua * r_ua;
                s_rs += -(double)delta * (double)inc;
                s_st += (double)inc * (double)inc;
                s_na += (double)ohi.v[c] * (double)ohi.v[c];
            }
            *reinterpret_cast<V*>(Ahi_out + off) = ohi;
            *reinterpret_cast<V*>(D0g + off) = dm;
            sOhi[i] = ohi;
            sD0[i] = dm;
            if constexpr (FF) {
                *reinterpret_cast<VF*>(Alo_out + off) = olo;
                sOlo[i] = olo;
            }
        }
        __syncthreads();

        // ---- edge phase: per-edge ||b_m||^2 and ||V_y - B_m||^2 on this slice
        for (int e = tid; e < m; e += kSliceThreads) {
            const int u = __ldg(P.ei + e), v = __ldg(P.ej + e);
            const R ta = onepb * __ldg(tm + e);
            const R tb = beta * __ldg(tm1 + e);
            const V hu = sOhi[u], hv = sOhi[v];
            const V mu_ = sD0[u], mv = sD0[v];
            const V pu = sD1[u], pv = sD1[v];
            VF lu, lv;
            if constexpr (FF) {
                lu = sOlo[u];
                lv = sOlo[v];
            }
            R sb = (R)0, sv = (R)0;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                R b = hu.v[c] - hv.v[c];
                if constexpr (FF) b += lu.v[c] - lv.v[c];
                const R dmv = mu_.v[c] - mv.v[c];
                const R d1v = pu.v[c] - pv.v[c];
                const R b1 = b - dmv;                   // b_{m-1}
                const R b2 = b1 - d1v;                  // b_{m-2}
                const R Dd = dmv - beta * d1v;          // delta_i - delta_j
                const R vmb = -Dd - (ta * b1 - tb * b2);
                sb += b * b;
                sv += vmb * vmb;
            }
            sNb[e] += (double)sb;
            s_vb += (double)sv;
        }
        __syncthreads();
    }

    // ---- partials of this CTA
    for (int e = tid; e < m; e += kSliceThreads) P.Pnb[(size_t)blockIdx.x * m + e] = sNb[e];
    double* ps = P.Ps + (size_t)blockIdx.x * kNumScalarPartials;
    double r;
    r = block_sum(s_ua, red);
    if (tid == 0) ps[kPsUA] = r;
    r = block_sum(s_vb, red);
    if (tid == 0) ps[kPsVB] = r;
    r = block_sum(s_rs, red);
    if (tid == 0) ps[kPsRestart] = r;
    r = block_sum(s_st, red);
    if (tid == 0) ps[kPsStep] = r;
    r = block_sum(s_na, red);
    if (tid == 0) ps[kPsNormA] = r;
    r = block_sum(s_nz, red);
    if (tid == 0) ps[kPsNoise] = r;
    r = block_sum(s_dl, red);
    if (tid == 0) ps[kPsDelta] = r;
}

// ------------------------------------------------------------------ reduce
template <typename R>
__global__ void __launch_bounds__(kReduceThreads) pd_reduce_kernel(IterParams<R> P) {
    PdState* st = P.st;
    if (st->done) return;
    __shared__ double s_d;
    __shared__ double red[32];
    __shared__ bool s_last;
    const int G = P.G, m = P.m, tid = threadIdx.x;
    if (tid == 0) {
        double acc = 0.0;
        for (int g = 0; g < G; ++g)
            acc += P.Ps[(size_t)g * kNumScalarPartials + kPsUA] + P.Ps[(size_t)g * kNumScalarPartials + kPsVB];
        s_d = sqrt(acc + st->eps);            // d_m (Eq. 5)
    }
    __syncthreads();
    const double d = s_d;
    const double gamma = st->gamma, rho = st->rho;
    R* tout = P.t[st->par ^ 1];              // t_{m+1} replaces t_{m-1}
    double cnt = 0.0;
    unsigned long long hsh = 0ULL;
    for (int e = blockIdx.x * blockDim.x + tid; e < m; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += P.Pnb[(size_t)g * m + e];
        const double nb = sqrt(s);
        const double lhs = gamma * P.w[e] * d;
        const double rhs = rho * nb;
        const bool fz = lhs >= rhs;          // prox returns exactly zero
        tout[e] = fz ? (R)1 : (R)(lhs / rhs);
        P.nb[e] = nb;
        P.fused[e] = fz ? 1 : 0;
        if (fz) {
            cnt += 1.0;
            hsh += mix64((unsigned long long)e + 1ULL);
        }
    }
    // fused count is exact in double; the hash is summed with wrap-around
    const double bc = block_sum(cnt, red);
    __shared__ unsigned long long sh[kReduceThreads];
    sh[tid] = hsh;
    __syncthreads();
    if (tid == 0) {
        unsigned long long hb = 0ULL;
        for (int k = 0; k < blockDim.x; ++k) hb += sh[k];
        P.Rf[2 * blockIdx.x] = (unsigned long long)bc;
        P.Rf[2 * blockIdx.x + 1] = hb;
        __threadfence();
        const unsigned int ticket = atomicAdd(&st->counter, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last || tid != 0) return;
    __threadfence();

    // ---- last block: scalar state update (serial, fixed order)
    unsigned long long nf = 0ULL, hash = 0ULL;
    for (int b = 0; b < (int)gridDim.x; ++b) {
        nf += P.Rf[2 * b];
        hash += P.Rf[2 * b + 1];
    }
    double rs = 0.0, stp = 0.0, na = 0.0, nzs = 0.0, dls = 0.0;
    for (int g = 0; g < G; ++g) {
        const double* ps = P.Ps + (size_t)g * kNumScalarPartials;
        rs += ps[kPsRestart];
        stp += ps[kPsStep];
        na += ps[kPsNormA];
        nzs += ps[kPsNoise];
        dls += ps[kPsDelta];
    }
    const double unit = sizeof(R) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
    const double noise = unit * sqrt(nzs);
    st->iter += 1;
    st->d_last = d;
    st->alpha2 = st->alpha1;
    st->alpha1 = d / (d + rho);
    if (st->accelerate) {
        // adaptive restart (O'Donoghue-Candes gradient test) on the projection:
        // drop the momentum when <a_start - A_m, A_m - A_{m-1}> > 0
        if (rs > 0.0) st->k_mom = 0;
        else st->k_mom += 1;
        const int k = st->k_mom;
        st->beta = k >= 1 ? (double)(k - 1) / (double)(k + 2) : 0.0;
    } else {
        st->beta = 0.0;
    }
    if ((int)nf == st->n_fused && hash == st->fused_hash) st->fused_stable += 1;
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
    if (st->iter % kConvWindow == 0) {
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
        if (cur == 0.0) {
            est = 0.0;
        } else if (st->ring_len == kRateWindows && cur < st->ring[0]) {
            const double g = log(st->ring[0] / cur) / (double)(kRateWindows * kConvWindow);
            est = cur / (g * g) / scale;
        }
        st->err_est = est;
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
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)P.m; e += (size_t)gridDim.x * blockDim.x) {
        P.t[0][e] = (R)1;   // t = 1 - s with s = 0: V_0 = 0
        P.t[1][e] = (R)1;
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
    }
}

__global__ void pd_begin_gamma_kernel(PdState* st, double gamma, double rho, double eps, double tol, int max_iter,
                                      int accelerate, double scale_floor) {
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
    for (int q = 0; q < kRateWindows; ++q) st->ring[q] = 0.0;
    st->dmax = 0.0;
    st->counter = 0u;
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

template <typename R>
cudaError_t launch_slice(const IterParams<R>& P, size_t smem, cudaStream_t s) {
    auto kern = pd_slice_kernel<R>;
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

size_t pd_slice_smem_bytes(int n, int m, bool fp64) {
    const size_t rows = fp64 ? (size_t)n * 4 * C * sizeof(double) : (size_t)n * 6 * C * sizeof(float);
    return rows + (size_t)m * sizeof(double);
}

int reduce_blocks(int m) {
    int b = (m + kReduceThreads - 1) / kReduceThreads;
    if (b < 1) b = 1;
    if (b > 128) b = 128;
    return b;
}

template <typename R>
cudaError_t launch_pd_slice(const IterParams<R>& P, cudaStream_t s) {
    const size_t smem = pd_slice_smem_bytes(P.n, P.m, std::is_same<R, double>::value);
    count_launches(1);
    return launch_slice<R>(P, smem, s);
}

template <typename R>
cudaError_t launch_pd_reduce(const IterParams<R>& P, cudaStream_t s) {
    count_launches(1);
    pd_reduce_kernel<R><<<reduce_blocks(P.m), kReduceThreads, 0, s>>>(P);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pd_iteration(const IterParams<R>& P, cudaStream_t s) {
    cudaError_t e = launch_pd_slice<R>(P, s);
    if (e != cudaSuccess) return e;
    return launch_pd_reduce<R>(P, s);
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
                                  int max_iter, int accelerate, double scale_floor, cudaStream_t s) {
    count_launches(1);
    pd_begin_gamma_kernel<<<1, 1, 0, s>>>(P.st, gamma, rho, eps, tol, max_iter, accelerate, scale_floor);
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
template cudaError_t launch_pd_slice<float>(const IterParams<float>&, cudaStream_t);
template cudaError_t launch_pd_slice<double>(const IterParams<double>&, cudaStream_t);
template cudaError_t launch_pd_reduce<float>(const IterParams<float>&, cudaStream_t);
template cudaError_t launch_pd_reduce<double>(const IterParams<double>&, cudaStream_t);
template cudaError_t launch_pd_iteration<double>(const IterParams<double>&, cudaStream_t);
template cudaError_t launch_pd_init<float>(const IterParams<float>&, const float*, cudaStream_t);
template cudaError_t launch_pd_init<double>(const IterParams<double>&, const double*, cudaStream_t);
template cudaError_t launch_pd_begin_gamma<float>(const IterParams<float>&, double, double, double, double, int, int,
                                                  double, cudaStream_t);
template cudaError_t launch_pd_begin_gamma<double>(const IterParams<double>&, double, double, double, double, int, int,
                                                   double, cudaStream_t);
template cudaError_t launch_pd_finalize<float>(const IterParams<float>&, float*, int64_t, int, cudaStream_t);
template cudaError_t launch_pd_finalize<double>(const IterParams<double>&, float*, int64_t, int, cudaStream_t);

}  // namespace ccx
