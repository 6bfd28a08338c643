// Anderson mixing of the PD/MM map (an acceleration of the fixed-point
// iteration; the fixed point, and so the result, is the paper's: Methods, Eq. 5
// and the U- and V-update displays).
//
// While a gamma's mixing phase is on, the iteration kernels run the plain map
// (no momentum): from z_k = (A_k, t_k, alpha_k) they produce the map's output
// G_k = (A_k + delta_k, t_(k+1), alpha_(k+1)) and its residual r_k = G_k - z_k
// (delta_k is the projection correction, held in the Delta slot).  Type-II
// Anderson mixing then takes
//     gamma = argmin || r_k - dR gamma ||,   z_(k+1) = G_k - dG gamma,
// over the last m differences dR_j = r_(j+1) - r_j and dG_j = G_(j+1) - G_j,
// kept in rings (float: they are differences of nearby iterates).  The missing
// entries' offsets are not mixed; they stay relative to A.
//
// pd_aa_update_kernel: adds the newest differences to the rings, forms the
//   partial inner products, and (last block to arrive) solves the small normal
//   equations in double and decides the hand-over: the phase ends when an edge
//   fuses (the map is not smooth there and the mixing stalls), when the
//   residual stops falling (it has reached its floor), or after kAaBudget
//   iterations; the restart rule then continues from the map's last output
//   and its own stopping test, with a fresh rate estimate, decides convergence.
// pd_aa_mix_kernel: applies the mix to A (float-float), to t at its three sweep
//   positions, and to alpha, and records the step z_(k+1) - z_k.
// Both return at once outside a mixing phase.  Sums are in a fixed order.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "ccx_internal.h"

namespace ccx {
namespace {

constexpr int kAaThreads = 256;
constexpr int kAaWarps = kAaThreads / 32;

// four consecutive entries: the rows are n x ld with ld a multiple of 32, so the
// matrices split into aligned groups of four and every load is a vector load
template <typename T>
struct alignas(sizeof(T) * 4) Quad {
    T v[4];
};
// Partial inner products of the update, for kernels whose rings hold at most M
// entries (M = 8 or kAaMax: the history length picks the instantiation, so a
// short history does not carry the registers of a long one).
template <int M>
struct AaSlots {
    static_assert(M <= kAaMax, "ring bound above the state's history arrays");
    static constexpr int RR = 0;            // <dR_new, dR_j>, j = 0 .. M - 1
    static constexpr int Rr = M;            // <dR_j, r_k>
    static constexpr int NN = 2 * M;        // <dR_new, dR_new>
    static constexpr int Nr = 2 * M + 1;    // <dR_new, r_k>
    static constexpr int rr = 2 * M + 2;    // <r_k, r_k>
    static constexpr int D = 2 * M + 3;     // number of partial sums (<= kAaDots)
};

__device__ __forceinline__ double aa_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void aa_ff_add(float hi, float lo, float inc, float& ohi, float& olo) {
    const float s = __fadd_rn(hi, inc);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(inc, bb));
    const float l = __fadd_rn(lo, err);
    const float h2 = __fadd_rn(s, l);
    olo = __fsub_rn(l, __fsub_rn(h2, s));
    ohi = h2;
}

// acc (hi + lo) += a * b without rounding the product (p + e = a b exactly, by
// an FMA) and with a compensated sum: about 48 bits, on the FP32 pipe
__device__ __forceinline__ void ff_dot(float a, float b, float& hi, float& lo) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float s = hi + p;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += err + e;
}

// ring slot j held a difference before this update: it lies within the last
// `len` slots before `head` (cyclically), and is not the slot being replaced
__device__ __forceinline__ bool aa_old_valid(int j, int m, int len, int head) {
    if (j >= m) return false;
    const int back = (head - 1 - j + m) % m;
    return back < len && j != head;
}

// The last block's thread 0: the alpha parts of the differences, the Gram
// matrix of the residual differences, the mixing coefficients (normal
// equations with a small ridge, Cholesky in double) and the hand-over test.
template <int M>
__device__ void aa_finish(PdState* st, const double* tot, const bool* old, int m, int len, int head, bool have) {
    using S = AaSlots<M>;
    const double ra = st->alpha1 - st->alpha2;   // alpha part of r_k (the reduction set alpha1 = G_k, alpha2 = z_k)
    const double rr = tot[S::rr] + ra * ra;
    int nlen = len, nhead = head;
    double g[M];
    for (int j = 0; j < M; ++j) g[j] = 0.0;
    if (have) {
        const double dn = ra - st->aa_ra_prev;
        double rR[M], Rr[M];
        for (int j = 0; j < M; ++j) {
            rR[j] = tot[S::RR + j];
            Rr[j] = tot[S::Rr + j];
            if (old[j]) {
                rR[j] += dn * st->aa_RA[j];
                Rr[j] += st->aa_RA[j] * ra;
            }
        }
        const double nn = tot[S::NN] + dn * dn, nr = tot[S::Nr] + dn * ra;
        st->aa_RA[head] = dn;
        st->aa_GA[head] = st->aa_sa + dn;
        for (int j = 0; j < M; ++j)
            if (old[j]) {
                st->aa_M[head][j] = rR[j];
                st->aa_M[j][head] = rR[j];
            }
        st->aa_M[head][head] = nn;
        // slots held after the update, oldest first
        nlen = len + 1 < m ? len + 1 : m;
        int idx[M];
        for (int a = 0; a < nlen; ++a) idx[a] = (head - (nlen - 1 - a) + m) % m;
        double A[M][M], b[M], y[M];
        double tr = 0.0;
        for (int a = 0; a < nlen; ++a) {
            b[a] = idx[a] == head ? nr : Rr[idx[a]];
            for (int c = 0; c < nlen; ++c) A[a][c] = st->aa_M[idx[a]][idx[c]];
            tr += A[a][a];
        }
        bool ok = tr > 0.0;
        const double lam = 1e-10 * tr / nlen;
        for (int a = 0; a < nlen; ++a) A[a][a] += lam;
        for (int c = 0; c < nlen && ok; ++c) {   // Cholesky: A = L L^T in the lower triangle
            double s = A[c][c];
            for (int q = 0; q < c; ++q) s -= A[c][q] * A[c][q];
            if (!(s > 0.0)) {
                ok = false;
                break;
            }
            A[c][c] = sqrt(s);
            for (int r2 = c + 1; r2 < nlen; ++r2) {
                double t = A[r2][c];
                for (int q = 0; q < c; ++q) t -= A[r2][q] * A[c][q];
                A[r2][c] = t / A[c][c];
            }
        }
        if (ok) {
            for (int a = 0; a < nlen; ++a) {
                double t = b[a];
                for (int q = 0; q < a; ++q) t -= A[a][q] * y[q];
                y[a] = t / A[a][a];
            }
            for (int a = nlen - 1; a >= 0; --a) {
                double t = y[a];
                for (int q = a + 1; q < nlen; ++q) t -= A[q][a] * y[q];
                y[a] = t / A[a][a];
            }
            double s1 = 0.0;
            for (int a = 0; a < nlen; ++a) s1 += fabs(y[a]);
            ok = s1 <= 1e4;                      // also false for a NaN
        }
        if (ok) {
            for (int a = 0; a < nlen; ++a) g[idx[a]] = y[a];
            nhead = (head + 1) % m;
        } else {
            nlen = 0;                            // the history starts again
            nhead = 0;
        }
    }
    for (int j = 0; j < M; ++j) st->aa_g[j] = g[j];
    st->aa_len = nlen;
    st->aa_head = nhead;
    st->aa_ra_prev = ra;
    st->aa_have_prev = 1;
    st->aa_iters += 1;
    st->aa_total += 1;
    // hand-over: a fused edge (the map is not smooth there), a residual that
    // stopped falling (no 2x over three windows), or the budget
    const double rn = sqrt(rr);
    bool stagnant = false;
    if (st->aa_iters % kConvWindow == 0) {
        for (int q = 0; q < 3; ++q) st->aa_win[q] = st->aa_win[q + 1];
        st->aa_win[3] = rn;
        stagnant = st->aa_iters >= 5 * kConvWindow && rn > 0.5 * st->aa_win[0];
    }
    if (st->n_fused > 0 || st->aa_iters >= kAaBudget || stagnant) {
        st->aa_on = 0;
        for (int j = 0; j < M; ++j) st->aa_g[j] = 0.0;
        // the restart rule takes over from the map's last output with a fresh
        // momentum and a fresh rate estimate for its stopping test
        st->k_mom = 0;
        st->beta = 0.0;
        st->ring_len = 0;
        for (int q = 0; q < kRateWindows; ++q) st->ring[q] = 0.0;
        st->dmax = 0.0;
        st->blk_max = 0.0;
        st->noise_max = 0.0;
        st->hits = 0;
        st->floor_hits = 0;
        st->stall_hits = 0;
        st->g_last = 0.0;
    }
    st->aa_counter = 0u;
}

template <typename R, int M>
__global__ void __launch_bounds__(kAaThreads) pd_aa_update_kernel(IterParams<R> P) {
    using S = AaSlots<M>;
    PdState* st = P.st;
    if (st->done || !st->aa_on) return;
    const int m = st->aa_m, len = st->aa_len, head = st->aa_head, par = st->par;
    const bool have = st->aa_have_prev != 0;
    const int LA = P.la * kSliceThreads, LE = P.le * kSliceThreads;
    const size_t NL = (size_t)P.n * P.ld;
    const R* __restrict__ rk = P.Dl[par];          // r_k (A part): this iteration's correction
    const R* __restrict__ rp = P.Dl[par ^ 1];      // r_(k-1)
    const R* __restrict__ tp = P.t[par] + 2 * (size_t)LA;   // (t_(k+1), t_k) at edge-sweep positions

    // a thread's own products in float-float (the normal equations of the mixing
    // are ill-conditioned: successive residual differences are nearly parallel),
    // the blocks' sums in double
    float fhi[S::D], flo[S::D];
#pragma unroll
    for (int q = 0; q < S::D; ++q) fhi[q] = flo[q] = 0.f;
    double acc[S::D];
    bool old[M];
#pragma unroll
    for (int j = 0; j < M; ++j) old[j] = have && aa_old_valid(j, m, len, head);

    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t NL4 = NL / 4;
    const Quad<R>* __restrict__ rk4 = reinterpret_cast<const Quad<R>*>(rk);
    const Quad<R>* __restrict__ rp4 = reinterpret_cast<const Quad<R>*>(rp);
    Quad<float>* __restrict__ R4 = reinterpret_cast<Quad<float>*>(P.aaR);
    Quad<float>* __restrict__ G4 = reinterpret_cast<Quad<float>*>(P.aaG);
    const Quad<float>* __restrict__ S4 = reinterpret_cast<const Quad<float>*>(P.aaS);
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < NL4; k += stride) {
        const Quad<R> r4 = rk4[k];
        if (!have) {
#pragma unroll
            for (int c = 0; c < 4; ++c) ff_dot((float)r4.v[c], (float)r4.v[c], fhi[S::rr], flo[S::rr]);
            continue;
        }
        const Quad<R> p4 = rp4[k];
        const Quad<float> s4 = S4[k];
        Quad<float> old4[M];
#pragma unroll
        for (int j = 0; j < M; ++j)
            if (old[j]) old4[j] = R4[(size_t)j * NL4 + k];
        Quad<float> nr4, ng4;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float r = (float)r4.v[c];
            const float dn = (float)((double)r4.v[c] - (double)p4.v[c]);
#pragma unroll
            for (int j = 0; j < M; ++j) {
                if (!old[j]) continue;
                const float Rj = old4[j].v[c];
                ff_dot(dn, Rj, fhi[S::RR + j], flo[S::RR + j]);
                ff_dot(Rj, r, fhi[S::Rr + j], flo[S::Rr + j]);
            }
            ff_dot(dn, dn, fhi[S::NN], flo[S::NN]);
            ff_dot(dn, r, fhi[S::Nr], flo[S::Nr]);
            ff_dot(r, r, fhi[S::rr], flo[S::rr]);
            nr4.v[c] = dn;
            ng4.v[c] = s4.v[c] + dn;
        }
        R4[(size_t)head * NL4 + k] = nr4;
        G4[(size_t)head * NL4 + k] = ng4;
    }
#pragma unroll
    for (int q = 0; q < S::D; ++q) acc[q] = (double)fhi[q] + (double)flo[q];
    for (size_t pos = blockIdx.x * (size_t)blockDim.x + threadIdx.x; pos < (size_t)LE; pos += stride) {
        if (P.eid[pos] < 0) continue;
        const double r = (double)tp[2 * pos] - (double)tp[2 * pos + 1];
        acc[S::rr] += r * r;
        if (have) {
            const double dn = r - (double)P.aaPt[pos];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                if (!old[j]) continue;
                const double Rj = (double)P.aaRt[(size_t)j * LE + pos];
                acc[S::RR + j] += dn * Rj;
                acc[S::Rr + j] += Rj * r;
            }
            acc[S::NN] += dn * dn;
            acc[S::Nr] += dn * r;
            P.aaRt[(size_t)head * LE + pos] = (float)dn;
            P.aaGt[(size_t)head * LE + pos] = (float)((double)P.aaSt[pos] + dn);
        }
        P.aaPt[pos] = (float)r;
    }

    // block sums in a fixed order: a shuffle tree per warp, then the warps in order
    __shared__ double red[kAaWarps][S::D];
    __shared__ double tot[S::D];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < S::D; ++q) {
        const double v = aa_warp_sum(acc[q]);
        if (lane == 0) red[wid][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < S::D) {
        double v = 0.0;
        for (int w = 0; w < kAaWarps; ++w) v += red[w][threadIdx.x];
        P.aaP[(size_t)blockIdx.x * S::D + threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int ticket = atomicAdd(&st->aa_counter, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the blocks' partials: thread t takes blocks t, t + 256, ..., then a fixed-order block sum
#pragma unroll
    for (int q = 0; q < S::D; ++q) acc[q] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < S::D; ++q) acc[q] += P.aaP[(size_t)b * S::D + q];
#pragma unroll
    for (int q = 0; q < S::D; ++q) {
        const double v = aa_warp_sum(acc[q]);
        if (lane == 0) red[wid][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < S::D) {
        double v = 0.0;
        for (int w = 0; w < kAaWarps; ++w) v += red[w][threadIdx.x];
        tot[threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // (continued in aa_finish: the last block's thread 0 solves and decides)
    aa_finish<M>(st, tot, old, m, len, head, have);
}

template <typename R, int M>
__global__ void __launch_bounds__(kAaThreads) pd_aa_mix_kernel(IterParams<R> P) {
    PdState* st = P.st;
    if (st->done || !st->aa_on) return;
    constexpr bool FF = std::is_same<R, float>::value;
    const int m = st->aa_m, par = st->par;
    const int LA = P.la * kSliceThreads, LE = P.le * kSliceThreads;
    const size_t NL = (size_t)P.n * P.ld;
    double g[M];
    float gf[M];
    bool use[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        g[j] = j < m ? st->aa_g[j] : 0.0;
        gf[j] = (float)g[j];
        use[j] = g[j] != 0.0;
    }
    Quad<R>* __restrict__ hi4 = reinterpret_cast<Quad<R>*>(P.Ahi[par]);   // G_k (A part), mixed into z_(k+1)
    Quad<float>* __restrict__ lo4 = reinterpret_cast<Quad<float>*>(P.Alo[par]);
    const Quad<R>* __restrict__ rk4 = reinterpret_cast<const Quad<R>*>(P.Dl[par]);   // r_k
    const Quad<float>* __restrict__ G4 = reinterpret_cast<const Quad<float>*>(P.aaG);
    Quad<float>* __restrict__ S4 = reinterpret_cast<Quad<float>*>(P.aaS);
    bool any = false;
#pragma unroll
    for (int j = 0; j < M; ++j) any = any || use[j];
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t NL4 = NL / 4;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < NL4; k += stride) {
        // the correction c = dG gamma in float: the mixed point only has to be close
        // to the best combination, the map evaluated at it fixes the result
        const Quad<R> r4 = rk4[k];
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        if (any) {
            Quad<float> gq[M];
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (use[j]) gq[j] = G4[(size_t)j * NL4 + k];
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (use[j])
#pragma unroll
                    for (int q = 0; q < 4; ++q) c[q] = fmaf(gf[j], gq[j].v[q], c[q]);
            Quad<R> h4 = hi4[k];
            if constexpr (FF) {
                Quad<float> l4 = lo4[k];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float h, l;
                    aa_ff_add(h4.v[q], l4.v[q], -c[q], h, l);
                    h4.v[q] = h;
                    l4.v[q] = l;
                }
                lo4[k] = l4;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) h4.v[q] -= (R)c[q];
            }
            hi4[k] = h4;
        }
        Quad<float> s4;
#pragma unroll
        for (int q = 0; q < 4; ++q) s4.v[q] = (float)r4.v[q] - c[q];   // z_(k+1) - z_k
        S4[k] = s4;
    }
    R* __restrict__ tp = P.t[par];
    for (size_t pos = blockIdx.x * (size_t)blockDim.x + threadIdx.x; pos < (size_t)LE; pos += stride) {
        if (P.eid[pos] < 0) continue;
        double c = 0.0;
#pragma unroll
        for (int j = 0; j < M; ++j)
            if (use[j]) c += g[j] * (double)P.aaGt[(size_t)j * LE + pos];
        const size_t e2 = 2 * (size_t)LA + 2 * pos;
        double tm = (double)tp[e2] - c;
        tm = tm < 0.0 ? 0.0 : (tm > 1.0 ? 1.0 : tm);
        P.aaSt[pos] = (float)(tm - (double)tp[e2 + 1]);
        const R tv = (R)tm;
        tp[e2] = tv;                               // edge-sweep position, then the two node-sweep ones
        const int2 qp = P.posA[pos];
        tp[2 * (size_t)qp.x] = tv;
        tp[2 * (size_t)qp.y] = tv;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double c = 0.0;
        for (int j = 0; j < M; ++j)
            if (use[j]) c += g[j] * st->aa_GA[j];
        double a1 = st->alpha1 - c;
        a1 = a1 < 0.0 ? 0.0 : (a1 >= 1.0 ? st->alpha1 : a1);
        st->aa_sa = a1 - st->alpha2;
        st->alpha1 = a1;
    }
}

}  // namespace

template <typename R>
cudaError_t launch_pd_aa(const IterParams<R>& P, cudaStream_t s) {
    if (!P.aaR || P.aa_blocks < 1) return cudaSuccess;   // no mixing buffers: mixing is off for this problem
    if (P.aa_hist < 1 || P.aa_hist > kAaMax) return cudaErrorInvalidValue;
    count_launches(2);
    if (P.aa_hist <= 8) {
        pd_aa_update_kernel<R, 8><<<P.aa_blocks, kAaThreads, 0, s>>>(P);
    } else {
        pd_aa_update_kernel<R, kAaMax><<<P.aa_blocks, kAaThreads, 0, s>>>(P);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (P.aa_hist <= 8) {
        pd_aa_mix_kernel<R, 8><<<P.aa_blocks, kAaThreads, 0, s>>>(P);
    } else {
        pd_aa_mix_kernel<R, kAaMax><<<P.aa_blocks, kAaThreads, 0, s>>>(P);
    }
    return cudaGetLastError();
}

template cudaError_t launch_pd_aa<float>(const IterParams<float>&, cudaStream_t);
template cudaError_t launch_pd_aa<double>(const IterParams<double>&, cudaStream_t);

}  // namespace ccx
