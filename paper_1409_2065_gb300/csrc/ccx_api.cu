// C ABI of the convex-clustering solver (include/ccx.h) and its host runtime:
// input validation; device buffers; the work layout of the iteration kernel
// (plan_sweeps); the warm-started gamma path as a resumable runner driving
// captured CUDA graphs of MM iterations, with the predictor between gammas and
// per-gamma outputs and labels; the batch driver and the serving scheduler
// built on the same runner; the kNN, connectivity and principal-axis entry
// points.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "ccx_internal.h"

namespace ccx {
void knn_set_exact_rows(const float* Xf, const uint32_t* bits, const double* colmean, int ldw);
}  // namespace ccx

using namespace ccx;

namespace {
std::atomic<unsigned long long> g_launches{0};
}  // namespace

void ccx::count_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {

thread_local std::string g_err;

ccx_status fail(ccx_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CUDA_TRY(expr)                                                                          \
    do {                                                                                        \
        cudaError_t _e = (expr);                                                                \
        if (_e != cudaSuccess) {                                                                \
            if (_e == cudaErrorMemoryAllocation)                                                \
                return fail(CCX_ENOMEM, "%s: %s", #expr, cudaGetErrorString(_e));               \
            return fail(CCX_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(_e));             \
        }                                                                                       \
    } while (0)

bool is_device_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count);
}

}  // namespace

namespace {
struct ShardState;
void drop_shard(ccx_problem* pr);
}  // namespace

struct ccx_problem {
    ShardState* shard = nullptr;  // feature-sharded iteration state (ccx_shard_*), created on first use
    int device = 0;
    cudaStream_t user = nullptr;
    cudaStream_t work = nullptr;
    cudaEvent_t ev_user = nullptr, ev_done = nullptr;
    cudaEvent_t ev_chunk[2] = {nullptr, nullptr};
    cudaEvent_t ev_out = nullptr;    // end of one gamma's output copies
    int precision = CCX_FP32;
    int64_t n = 0, p = 0, ld_in = 0;
    int ld = 0, ldw = 0, nslices = 0, G = 0, num_sms = 0;
    bool has_mask = false;
    // data
    float* Xf = nullptr;
    double* Xd = nullptr;
    uint32_t* maskbits = nullptr;
    double* colmean = nullptr;   // 2 * ld doubles (means, then per-column scratch)
    float* Y0f = nullptr;
    double* Y0d = nullptr;
    double* d_ss = nullptr;
    double nyc = 0.0;            // ||Y_c||_F
    double ny0 = 0.0;            // ||Y_0||_F
    // edges
    std::vector<int> ei, ej;
    std::vector<double> w;
    double nw = 0.0;             // ||w||_2
    int deg_max = 0;
    int* d_ei = nullptr;
    int* d_ej = nullptr;
    double* d_w = nullptr;
    int* d_rowptr = nullptr;
    int* d_erow = nullptr;
    int* d_ps0 = nullptr;
    uint16_t* d_csrT = nullptr;
    uint16_t* d_ejT = nullptr;
    uint2* d_thrA = nullptr;
    int* d_thrE = nullptr;
    int2* d_posA = nullptr;
    int* d_eid = nullptr;
    int la = 1, le = 1, nslots = 0;
    // path state
    void* A[2] = {nullptr, nullptr};
    float* Alo[2] = {nullptr, nullptr};
    void* Dl[2] = {nullptr, nullptr};
    void* Q = nullptr;
    void* Em = nullptr;
    void* t[2] = {nullptr, nullptr};
    float* Pnb = nullptr;
    double* Ps = nullptr;
    double* nb = nullptr;
    uint8_t* fused = nullptr;
    unsigned long long* Rf = nullptr;
    PdState* st = nullptr;
    PdState* st_host = nullptr;  // pinned, 2 slots
    float* Ustage = nullptr;
    int* Lstage = nullptr;
    int* cc_scratch = nullptr;
    int* d_ncl = nullptr;
    int* h_ncl = nullptr;        // pinned
    double* pc_axes = nullptr;   // q x p principal axes of Y_0 (device), computed on request
    int pc_q = 0;
    std::vector<double> pc_var;
    float* Sstage = nullptr;     // n x q projected scores (device staging for host outputs)
    void* Aprev = nullptr;       // A at the end of the previous gamma (hi, or double)
    float* Aprev_lo = nullptr;   // its lo part (FP32 path)
    void* Aprev2 = nullptr;      // A at the end of the gamma before that (quadratic predictor)
    float* Aprev2_lo = nullptr;
    bool path_ready = false;
    bool path_started = false;
    cudaGraphExec_t graph = nullptr;
    int graph_chunk = 0;
    int graph_stream = 0;        // stream_edges the captured graph was built with
    int graph_variant = -1;      // slice_variant, grid and fuse_delta the captured graph was built with
    int graph_G = 0;
    double graph_delta = -1.0;
    int stream_edges = 0;        // from the options of the current call
    int variant = 0;
    int max_ctas = 0;
    int tuned_G = 0;             // grid chosen by ccx_tune_grid (0: none), used when the options set no cap
    double delta_fuse = 1e-5;
    // Anderson mixing (opts.anderson): history length of the current call, the one the
    // buffers were sized for, the one the captured graph was built with, and the buffers
    int aa_use = 0, aa_alloc = 0, graph_aa = -1;
    float* aaR = nullptr;
    float* aaG = nullptr;
    float* aaS = nullptr;
    float* aaRt = nullptr;
    float* aaGt = nullptr;
    float* aaSt = nullptr;
    float* aaPt = nullptr;
    double* aaP = nullptr;
    int last_fused = -1;         // fused edges at the end of the last solved gamma (-1: none yet)
};

namespace {

void free_path(ccx_problem* pr) {
    for (int k = 0; k < 2; ++k) {
        cudaFree(pr->A[k]);
        cudaFree(pr->Alo[k]);
        cudaFree(pr->Dl[k]);
        cudaFree(pr->t[k]);
        pr->A[k] = pr->Alo[k] = nullptr;
        pr->Dl[k] = pr->t[k] = nullptr;
    }
    cudaFree(pr->Q);
    cudaFree(pr->Em);
    cudaFree(pr->Aprev);
    cudaFree(pr->Aprev_lo);
    cudaFree(pr->Aprev2);
    cudaFree(pr->Aprev2_lo);
    pr->Aprev = pr->Aprev2 = nullptr;
    pr->Aprev_lo = pr->Aprev2_lo = nullptr;
    cudaFree(pr->aaR);
    cudaFree(pr->aaG);
    cudaFree(pr->aaS);
    cudaFree(pr->aaRt);
    cudaFree(pr->aaGt);
    cudaFree(pr->aaSt);
    cudaFree(pr->aaPt);
    cudaFree(pr->aaP);
    pr->aaR = pr->aaG = pr->aaS = pr->aaRt = pr->aaGt = pr->aaSt = pr->aaPt = nullptr;
    pr->aaP = nullptr;
    pr->aa_alloc = 0;
    pr->last_fused = -1;
    cudaFree(pr->Pnb);
    cudaFree(pr->Ps);
    cudaFree(pr->nb);
    cudaFree(pr->fused);
    cudaFree(pr->Rf);
    cudaFree(pr->st);
    cudaFree(pr->Ustage);
    cudaFree(pr->Lstage);
    cudaFree(pr->cc_scratch);
    cudaFree(pr->d_ncl);
    if (pr->st_host) cudaFreeHost(pr->st_host);
    if (pr->h_ncl) cudaFreeHost(pr->h_ncl);
    if (pr->graph) cudaGraphExecDestroy(pr->graph);
    pr->Q = pr->Em = nullptr;
    pr->Pnb = nullptr;
    pr->Ps = pr->nb = nullptr;
    pr->fused = nullptr;
    pr->Rf = nullptr;
    pr->st = nullptr;
    pr->st_host = nullptr;
    pr->Ustage = nullptr;
    pr->Lstage = pr->cc_scratch = pr->d_ncl = pr->h_ncl = nullptr;
    pr->graph = nullptr;
    pr->graph_chunk = 0;
    pr->path_ready = false;
    pr->path_started = false;
}

void free_edges(ccx_problem* pr) {
    cudaFree(pr->d_ei);
    cudaFree(pr->d_ej);
    cudaFree(pr->d_w);
    cudaFree(pr->d_rowptr);
    cudaFree(pr->d_erow);
    cudaFree(pr->d_ps0);
    cudaFree(pr->d_csrT);
    cudaFree(pr->d_ejT);
    cudaFree(pr->d_thrA);
    cudaFree(pr->d_thrE);
    cudaFree(pr->d_posA);
    cudaFree(pr->d_eid);
    pr->d_eid = nullptr;
    pr->d_ei = pr->d_ej = pr->d_rowptr = pr->d_erow = pr->d_ps0 = pr->d_thrE = nullptr;
    pr->d_csrT = pr->d_ejT = nullptr;
    pr->d_thrA = nullptr;
    pr->d_posA = nullptr;
    pr->d_w = nullptr;
}

void free_all(ccx_problem* pr) {
    free_path(pr);
    free_edges(pr);
    cudaFree(pr->Xf);
    cudaFree(pr->Xd);
    cudaFree(pr->maskbits);
    cudaFree(pr->colmean);
    cudaFree(pr->Y0f);
    cudaFree(pr->pc_axes);
    cudaFree(pr->Sstage);
    cudaFree(pr->Y0d);
    cudaFree(pr->d_ss);
    if (pr->ev_user) cudaEventDestroy(pr->ev_user);
    if (pr->ev_done) cudaEventDestroy(pr->ev_done);
    for (int k = 0; k < 2; ++k)
        if (pr->ev_chunk[k]) cudaEventDestroy(pr->ev_chunk[k]);
    if (pr->ev_out) cudaEventDestroy(pr->ev_out);
    if (pr->work) cudaStreamDestroy(pr->work);
}

// make the work stream wait for everything already queued on the caller's stream
ccx_status enter(ccx_problem* pr) {
    CUDA_TRY(cudaSetDevice(pr->device));
    CUDA_TRY(cudaEventRecord(pr->ev_user, pr->user));
    CUDA_TRY(cudaStreamWaitEvent(pr->work, pr->ev_user, 0));
    return CCX_OK;
}

// make the caller's stream wait for the work and wait on the host
ccx_status leave(ccx_problem* pr) {
    CUDA_TRY(cudaEventRecord(pr->ev_done, pr->work));
    CUDA_TRY(cudaStreamWaitEvent(pr->user, pr->ev_done, 0));
    CUDA_TRY(cudaStreamSynchronize(pr->work));
    return CCX_OK;
}

// Order of the entries inside the runs of one sweep.  A sweep's N entries
// (0..N-1) are cut into T runs of L consecutive entries; entry x gathers the
// shared-memory row of node val[x] and belongs to segment seg[x] (its row).
// Within a run the entries of one segment may be taken in any order.  128-bit
// shared loads are served eight lanes at a time, and lanes whose rows fall in
// the same 16-byte bank group (node mod ncol) are served one after another, so
// at every step the eight runs of each group of lanes are given rows in
// distinct bank groups where their segments allow it (a bipartite matching of
// lanes to bank groups per step).  Returns at[k*T + t] = entry taken by run t at
// step k (-1 past the end).
std::vector<int64_t> arrange_runs(int T, int L, int64_t N, const std::vector<int>& val, const std::vector<int>& seg,
                                  int ncol) {
    std::vector<int64_t> at((size_t)L * T, -1);
    for (int g = 0; g < T; g += 8) {
        const int nl = std::min(8, T - g);
        std::vector<int64_t> next(nl), end(nl);     // next unstarted entry, end of the run
        std::vector<std::vector<int64_t>> rem(nl);  // remaining entries of the current segment
        for (int l = 0; l < nl; ++l) {
            next[l] = std::min<int64_t>((int64_t)(g + l) * L, N);
            end[l] = std::min<int64_t>(next[l] + L, N);
        }
        auto refill = [&](int l) {
            if (!rem[l].empty() || next[l] >= end[l]) return;
            const int64_t a = next[l];
            int64_t b = a;
            while (b < end[l] && seg[b] == seg[a]) ++b;
            for (int64_t x = a; x < b; ++x) rem[l].push_back(x);
            next[l] = b;
        };
        for (int k = 0; k < L; ++k) {
            std::vector<int> lanes;
            std::vector<std::vector<int>> cnt(nl, std::vector<int>(ncol, 0));
            for (int l = 0; l < nl; ++l) {
                refill(l);
                if (rem[l].empty()) continue;
                lanes.push_back(l);
                for (int64_t x : rem[l]) cnt[l][val[x] % ncol]++;
            }
            auto nopt = [&](int l) {
                int c = 0;
                for (int q = 0; q < ncol; ++q) c += cnt[l][q] > 0;
                return c;
            };
            std::stable_sort(lanes.begin(), lanes.end(), [&](int a, int b) { return nopt(a) < nopt(b); });
            std::vector<int> owner(ncol, -1), lane_col(nl, -1);
            std::function<bool(int, std::vector<char>&)> augment = [&](int l, std::vector<char>& seen) {
                std::vector<int> cols;
                for (int q = 0; q < ncol; ++q)
                    if (cnt[l][q] > 0) cols.push_back(q);
                std::stable_sort(cols.begin(), cols.end(), [&](int a, int b) { return cnt[l][a] > cnt[l][b]; });
                for (int q : cols) {
                    if (seen[q]) continue;
                    seen[q] = 1;
                    if (owner[q] < 0 || augment(owner[q], seen)) {
                        owner[q] = l;
                        lane_col[l] = q;
                        return true;
                    }
                }
                return false;
            };
            for (int l : lanes) {
                std::vector<char> seen(ncol, 0);
                augment(l, seen);
            }
            for (int l : lanes) {
                int q = lane_col[l];
                if (q < 0 || owner[q] != l) {   // unmatched: take the most common bank group
                    q = 0;
                    for (int c = 1; c < ncol; ++c)
                        if (cnt[l][c] > cnt[l][q]) q = c;
                }
                size_t pick = 0;
                while (val[rem[l][pick]] % ncol != q) ++pick;
                at[(size_t)k * T + g + l] = rem[l][pick];
                rem[l].erase(rem[l].begin() + (long)pick);
            }
        }
    }
    return at;
}

// The work layout of the iteration kernel's two sweeps for a sorted edge set
// (i < j, ordered by (i, j), no duplicates): CSR over both directions, the
// equal per-thread runs with their bank-aware order, partial slots and the
// position maps the reduction uses.  Host only.
struct SweepPlan {
    int la = 1, le = 1, nslots = 0, deg_max = 0;
    std::vector<int> rowptr, erow, ps0, thrE, eid, node_row;
    std::vector<uint16_t> csrT, ejT;
    std::vector<uint2> thrA;
    std::vector<int2> posE;
};

SweepPlan plan_sweeps(int64_t n, const std::vector<int>& ei, const std::vector<int>& ej, int precision) {
    SweepPlan P;
    const int m = (int)ei.size();
    std::vector<int> deg(n, 0);
    for (int q = 0; q < m; ++q) {
        deg[ei[q]]++;
        deg[ej[q]]++;
    }
    std::vector<int> rowptr(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) rowptr[i + 1] = rowptr[i] + deg[i];
    P.deg_max = n > 0 ? *std::max_element(deg.begin(), deg.end()) : 0;
    std::vector<std::pair<int, int>> ent(2 * (size_t)m);
    std::vector<int> fillp(rowptr.begin(), rowptr.end() - 1);
    for (int q = 0; q < m; ++q) {
        ent[fillp[ei[q]]++] = {ej[q], q};
        ent[fillp[ej[q]]++] = {ei[q], q};
    }
    // rows by increasing neighbour; qa/qb: CSR position of edge e in the row of ei / ej
    std::vector<uint16_t> csr(2 * (size_t)m);
    std::vector<int> qa(m), qb(m), rowof(2 * (size_t)m);
    for (int64_t i = 0; i < n; ++i) {
        std::sort(ent.begin() + rowptr[i], ent.begin() + rowptr[i + 1]);
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            csr[k] = (uint16_t)ent[k].first;
            rowof[k] = (int)i;
            (ent[k].first > i ? qa : qb)[ent[k].second] = k;
        }
    }
    // equal runs of the two sweeps, one per thread of the iteration kernel
    const int T = kSliceThreads;
    const int64_t m2 = 2 * (int64_t)m;
    const int la = (int)std::max<int64_t>(1, (m2 + T - 1) / T);
    const int le = std::max(1, (m + T - 1) / T);
    // bank groups of a node's shared row slice: 128 bytes / row bytes (8 for 16-byte rows, 4 for 32-byte)
    const int row_bytes = kSliceCols * (precision == CCX_FP64 ? 8 : 4);
    const int ncol = std::max(1, 128 / std::max(16, row_bytes));
    std::vector<int> csr_val(csr.begin(), csr.end());
    const std::vector<int64_t> atA = arrange_runs(T, la, m2, csr_val, rowof, ncol);
    const std::vector<int64_t> atE = arrange_runs(T, le, m, ej, ei, ncol);
    std::vector<int> posA_of(m2 > 0 ? m2 : 1);
    std::vector<uint16_t> csrT((size_t)la * T, 0), ejT((size_t)le * T, 0);
    for (size_t x = 0; x < atA.size(); ++x)
        if (atA[x] >= 0) {
            csrT[x] = csr[atA[x]];
            posA_of[atA[x]] = (int)x;
        }
    std::vector<int> eid((size_t)le * T, -1);
    std::vector<int2> posE((size_t)le * T, make_int2(0, 0));
    for (size_t x = 0; x < atE.size(); ++x)
        if (atE[x] >= 0) {
            const int e = (int)atE[x];
            ejT[x] = (uint16_t)ej[e];
            eid[x] = e;
            posE[x] = make_int2(posA_of[qa[e]], posA_of[qb[e]]);
        }
    // node-sweep partial slots: one per (run, row) overlap, numbered in entry
    // order, so the slots of a node are consecutive
    std::vector<uint2> thrA(T);
    std::vector<int> ps0(n + 1, 0);
    int nslots = 0;
    for (int t = 0; t < T; ++t) {
        const int64_t q0 = (int64_t)t * la, q1 = std::min<int64_t>(q0 + la, m2);
        thrA[t] = make_uint2(q0 < q1 ? (uint32_t)rowof[q0] : 0u, (uint32_t)nslots);
        for (int64_t q = q0; q < q1; ++q)
            if (q == q0 || rowof[q] != rowof[q - 1]) {
                ps0[rowof[q] + 1]++;
                ++nslots;
            }
    }
    for (int64_t i = 0; i < n; ++i) ps0[i + 1] += ps0[i];
    std::vector<int> erow(n + 1, 0), thrE(T, 0);
    for (int e = 0; e < m; ++e) erow[ei[e] + 1]++;
    for (int64_t i = 0; i < n; ++i) erow[i + 1] += erow[i];
    for (int t = 0; t < T; ++t)
        if ((int64_t)t * le < m) thrE[t] = ei[(size_t)t * le];
    P.node_row.assign((size_t)la * T, -1);
    for (size_t x = 0; x < atA.size(); ++x)
        if (atA[x] >= 0) P.node_row[x] = rowof[atA[x]];
    P.la = la;
    P.le = le;
    P.nslots = nslots;
    P.rowptr = std::move(rowptr);
    P.erow = std::move(erow);
    P.ps0 = std::move(ps0);
    P.thrE = std::move(thrE);
    P.eid = std::move(eid);
    P.csrT = std::move(csrT);
    P.ejT = std::move(ejT);
    P.thrA = std::move(thrA);
    P.posE = std::move(posE);
    return P;
}

// Validate, sort by (i, j), drop zero weights, store and upload with CSR.
ccx_status install_edges(ccx_problem* pr, const std::vector<int>& ei_in, const std::vector<int>& ej_in,
                         const std::vector<double>& w_in) {
    const int64_t n = pr->n;
    const size_t m0 = ei_in.size();
    std::vector<size_t> order;
    order.reserve(m0);
    for (size_t e = 0; e < m0; ++e) {
        const int64_t a = ei_in[e], b = ej_in[e];
        const double wt = w_in[e];
        if (a < 0 || b < 0 || a >= n || b >= n)
            return fail(CCX_EINVAL, "edge %zu: index out of range [0, %lld)", e, (long long)n);
        if (a >= b) return fail(CCX_EINVAL, "edge %zu: need ei < ej (got %lld, %lld)", e, (long long)a, (long long)b);
        if (!std::isfinite(wt) || wt < 0.0) return fail(CCX_EINVAL, "edge %zu: weight must be finite and >= 0", e);
        if (wt > 0.0) order.push_back(e);
    }
    std::sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        return ei_in[x] != ei_in[y] ? ei_in[x] < ei_in[y] : ej_in[x] < ej_in[y];
    });
    for (size_t q = 1; q < order.size(); ++q)
        if (ei_in[order[q]] == ei_in[order[q - 1]] && ej_in[order[q]] == ej_in[order[q - 1]])
            return fail(CCX_EINVAL, "duplicate edge (%d, %d)", ei_in[order[q]], ej_in[order[q]]);
    const int m = (int)order.size();
    pr->ei.resize(m);
    pr->ej.resize(m);
    pr->w.resize(m);
    double s2 = 0.0;
    for (int q = 0; q < m; ++q) {
        pr->ei[q] = ei_in[order[q]];
        pr->ej[q] = ej_in[order[q]];
        pr->w[q] = w_in[order[q]];
        s2 += pr->w[q] * pr->w[q];
    }
    pr->nw = std::sqrt(s2);
    // CSR over both directions; each row lists its neighbours by increasing index
    SweepPlan P = plan_sweeps(n, pr->ei, pr->ej, pr->precision);
    pr->deg_max = P.deg_max;
    const int T = kSliceThreads;
    const int la = P.la, le = P.le, nslots = P.nslots;
    std::vector<int>& rowptr = P.rowptr;
    std::vector<int>& erow = P.erow;
    std::vector<int>& ps0 = P.ps0;
    std::vector<int>& thrE = P.thrE;
    std::vector<int>& eid = P.eid;
    std::vector<uint16_t>& csrT = P.csrT;
    std::vector<uint16_t>& ejT = P.ejT;
    std::vector<uint2>& thrA = P.thrA;
    std::vector<int2>& posE = P.posE;
    free_path(pr);
    free_edges(pr);
    pr->la = la;
    pr->le = le;
    pr->nslots = nslots;
    CUDA_TRY(dalloc(&pr->d_ei, m));
    CUDA_TRY(dalloc(&pr->d_ej, m));
    CUDA_TRY(dalloc(&pr->d_w, m));
    CUDA_TRY(dalloc(&pr->d_rowptr, n + 1));
    CUDA_TRY(dalloc(&pr->d_erow, n + 1));
    CUDA_TRY(dalloc(&pr->d_ps0, n + 1));
    CUDA_TRY(dalloc(&pr->d_csrT, csrT.size()));
    CUDA_TRY(dalloc(&pr->d_ejT, ejT.size()));
    CUDA_TRY(dalloc(&pr->d_thrA, T));
    CUDA_TRY(dalloc(&pr->d_thrE, T));
    CUDA_TRY(dalloc(&pr->d_posA, posE.size()));
    CUDA_TRY(dalloc(&pr->d_eid, eid.size()));
    if (m > 0) {
        CUDA_TRY(cudaMemcpy(pr->d_ei, pr->ei.data(), sizeof(int) * m, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(pr->d_ej, pr->ej.data(), sizeof(int) * m, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(pr->d_w, pr->w.data(), sizeof(double) * m, cudaMemcpyHostToDevice));
    }
    CUDA_TRY(cudaMemcpy(pr->d_csrT, csrT.data(), sizeof(uint16_t) * csrT.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pr->d_ejT, ejT.data(), sizeof(uint16_t) * ejT.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pr->d_thrA, thrA.data(), sizeof(uint2) * T, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pr->d_thrE, thrE.data(), sizeof(int) * T, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pr->d_posA, posE.data(), sizeof(int2) * posE.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pr->d_eid, eid.data(), sizeof(int) * eid.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pr->d_rowptr, rowptr.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pr->d_erow, erow.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pr->d_ps0, ps0.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
    return CCX_OK;
}

template <typename R>
IterParams<R> make_params(ccx_problem* pr) {
    IterParams<R> P{};
    P.X = std::is_same<R, double>::value ? reinterpret_cast<const R*>(pr->Xd) : reinterpret_cast<const R*>(pr->Xf);
    P.mask = pr->has_mask ? pr->maskbits : nullptr;
    for (int k = 0; k < 2; ++k) {
        P.Ahi[k] = reinterpret_cast<R*>(pr->A[k]);
        P.Alo[k] = pr->Alo[k];
        P.Dl[k] = reinterpret_cast<R*>(pr->Dl[k]);
        P.t[k] = reinterpret_cast<R*>(pr->t[k]);
    }
    P.Q = reinterpret_cast<R*>(pr->Q);
    P.Em = reinterpret_cast<R*>(pr->Em);
    P.rowptr = pr->d_rowptr;
    P.erow = pr->d_erow;
    P.ps0 = pr->d_ps0;
    P.csrT = pr->d_csrT;
    P.ejT = pr->d_ejT;
    P.thrA = pr->d_thrA;
    P.thrE = pr->d_thrE;
    P.posA = pr->d_posA;
    P.eid = pr->d_eid;
    P.la = pr->la;
    P.le = pr->le;
    P.nslots = pr->nslots;
    P.stream_edges = pr->stream_edges;
    P.delta_fuse = pr->delta_fuse;
    P.ext_part = nullptr;
    P.n_ext = 0;
    P.ext_len = 0;
    P.p = (int)pr->p;
    const bool aa = pr->aa_use > 0 && pr->aa_alloc == pr->aa_use;
    P.aaR = aa ? pr->aaR : nullptr;
    P.aaG = aa ? pr->aaG : nullptr;
    P.aaS = aa ? pr->aaS : nullptr;
    P.aaRt = aa ? pr->aaRt : nullptr;
    P.aaGt = aa ? pr->aaGt : nullptr;
    P.aaSt = aa ? pr->aaSt : nullptr;
    P.aaPt = aa ? pr->aaPt : nullptr;
    P.aaP = aa ? pr->aaP : nullptr;
    // mixing kernels: four blocks per SM, or fewer when the matrix has fewer groups of
    // four entries than that many blocks have threads (small problems in a batch)
    const size_t aa_quads = (size_t)pr->n * pr->ld / 4;
    const size_t aa_need = (aa_quads + 255) / 256;
    P.aa_blocks = aa ? (int)std::max<size_t>(1, std::min<size_t>(aa_need, (size_t)4 * pr->num_sms)) : 0;
    P.aa_hist = aa ? pr->aa_use : 0;
    P.ei = pr->d_ei;
    P.ej = pr->d_ej;
    P.w = pr->d_w;
    P.Pnb = pr->Pnb;
    P.Ps = pr->Ps;
    P.nb = pr->nb;
    P.fused = pr->fused;
    P.Rf = pr->Rf;
    P.st = pr->st;
    P.n = (int)pr->n;
    P.ld = pr->ld;
    P.ldw = pr->ldw;
    P.m = (int)pr->ei.size();
    P.nslices = pr->nslices;
    P.G = pr->G;
    return P;
}

ccx_status check_limits(ccx_problem* pr) {
    const int m = (int)pr->ei.size();
    if (pr->n > 65535)
        return fail(CCX_EUNSUPPORTED, "the iteration kernel stores node indices in 16 bits: n must be <= 65535 "
                                      "(have %lld)", (long long)pr->n);
    int optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pr->device));
    // the smallest variant of the iteration kernel keeps only the rows of a slice in shared memory
    const size_t need = pd_slice_smem_bytes((int)pr->n, pr->la, pr->le, pr->nslots, pr->precision == CCX_FP64, false,
                                            true);
    if (need + 2048 > (size_t)optin)
        return fail(CCX_EUNSUPPORTED,
                    "n = %lld cases and %d edges need %zu bytes of shared memory per block (a column slice of "
                    "all rows and the partial sums of the node sweep); the device allows %d",
                    (long long)pr->n, m, need, optin);
    return CCX_OK;
}

// grid of the iteration kernel: one CTA per SM, at most one per slice, capped by `cap` (> 0)
int grid_of_cap(const ccx_problem* pr, int cap) {
    const int nsl = (int)((pr->p + kSliceCols - 1) / kSliceCols);
    int G = std::min(nsl, pr->num_sms);
    if (cap > 0) G = std::min(G, cap);
    return std::max(G, 1);
}

int grid_of(const ccx_problem* pr) { return grid_of_cap(pr, pr->max_ctas); }

// The options of a call that shape the iteration kernel's launch.
void apply_opts(ccx_problem* pr, const ccx_opts& o) {
    pr->stream_edges = o.stream_edges ? 1 : 0;
    pr->variant = o.slice_variant;
    pr->max_ctas = o.max_ctas > 0 ? o.max_ctas : pr->tuned_G;
    pr->delta_fuse = o.fuse_delta;
    pr->aa_use = o.anderson;
}

ccx_status ensure_path(ccx_problem* pr) {
    if (pr->path_ready) {
        // a changed grid cap resizes the per-CTA partial buffers (the path state is kept);
        // a captured iteration graph holds the old buffers' addresses, so it goes too
        const int G = grid_of(pr);
        if (G != pr->G) {
            if (pr->graph) {
                CUDA_TRY(cudaStreamSynchronize(pr->work));
                cudaGraphExecDestroy(pr->graph);
                pr->graph = nullptr;
                pr->graph_chunk = 0;
            }
            CUDA_TRY(cudaStreamSynchronize(pr->work));
            cudaFree(pr->Pnb);
            cudaFree(pr->Ps);
            pr->Pnb = nullptr;
            pr->Ps = nullptr;
            pr->G = G;
            CUDA_TRY(dalloc(&pr->Pnb, (size_t)G * pr->le * kSliceThreads));
            CUDA_TRY(dalloc(&pr->Ps, (size_t)G * kNumScalarPartials));
        }
        return CCX_OK;
    }
    const bool fp64 = pr->precision == CCX_FP64;
    const size_t es = fp64 ? sizeof(double) : sizeof(float);
    const size_t nl = (size_t)pr->n * pr->ld;
    const int m = (int)pr->ei.size();
    pr->nslices = (int)((pr->p + kSliceCols - 1) / kSliceCols);
    pr->G = grid_of(pr);
    for (int k = 0; k < 2; ++k) {
        CUDA_TRY(cudaMalloc(&pr->A[k], es * nl));
        CUDA_TRY(cudaMalloc(&pr->Dl[k], es * nl));
        if (!fp64) CUDA_TRY(dalloc(&pr->Alo[k], nl));
        if (k == 0) {
            CUDA_TRY(cudaMalloc(&pr->Aprev, es * nl));
            if (!fp64) CUDA_TRY(dalloc(&pr->Aprev_lo, nl));
        }
        // a (t, t_prev) pair per node-sweep and per edge-sweep position
        CUDA_TRY(cudaMalloc(&pr->t[k], es * 2 * ((size_t)pr->la + pr->le) * kSliceThreads));
    }
    if (pr->has_mask) {
        CUDA_TRY(cudaMalloc(&pr->Q, es * nl));
        CUDA_TRY(cudaMalloc(&pr->Em, es * nl));
    }
    CUDA_TRY(dalloc(&pr->Pnb, (size_t)pr->G * pr->le * kSliceThreads));
    CUDA_TRY(dalloc(&pr->Ps, (size_t)pr->G * kNumScalarPartials));
    CUDA_TRY(dalloc(&pr->nb, m));
    CUDA_TRY(dalloc(&pr->fused, m));
    CUDA_TRY(dalloc(&pr->Rf, 3 * (size_t)pd_reduce_blocks(pr->le)));
    CUDA_TRY(dalloc(&pr->st, 1));
    CUDA_TRY(cudaMallocHost(&pr->st_host, 2 * sizeof(PdState)));
    CUDA_TRY(dalloc(&pr->Ustage, (size_t)pr->n * pr->p));
    CUDA_TRY(dalloc(&pr->Lstage, pr->n));
    CUDA_TRY(dalloc(&pr->cc_scratch, pr->n));
    CUDA_TRY(dalloc(&pr->d_ncl, 1));
    CUDA_TRY(cudaMallocHost(&pr->h_ncl, sizeof(int)));
    CUDA_TRY(cudaMemsetAsync(pr->st, 0, sizeof(PdState), pr->work));
    pr->path_ready = true;
    pr->path_started = false;
    return CCX_OK;
}

// Buffers of the Anderson mixing for history aa_use (sized once per length; a
// change drops the captured graph, which holds their addresses).
ccx_status ensure_aa(ccx_problem* pr) {
    const int m = pr->aa_use;
    if (m <= 0 || pr->aa_alloc == m) return CCX_OK;
    if (pr->graph) {
        CUDA_TRY(cudaStreamSynchronize(pr->work));
        cudaGraphExecDestroy(pr->graph);
        pr->graph = nullptr;
        pr->graph_chunk = 0;
    }
    CUDA_TRY(cudaStreamSynchronize(pr->work));
    cudaFree(pr->aaR);
    cudaFree(pr->aaG);
    cudaFree(pr->aaS);
    cudaFree(pr->aaRt);
    cudaFree(pr->aaGt);
    cudaFree(pr->aaSt);
    cudaFree(pr->aaPt);
    cudaFree(pr->aaP);
    pr->aaR = pr->aaG = pr->aaS = pr->aaRt = pr->aaGt = pr->aaSt = pr->aaPt = nullptr;
    pr->aaP = nullptr;
    pr->aa_alloc = 0;
    const size_t nl = (size_t)pr->n * pr->ld;
    const size_t LE = (size_t)pr->le * kSliceThreads;
    CUDA_TRY(dalloc(&pr->aaR, (size_t)m * nl));
    CUDA_TRY(dalloc(&pr->aaG, (size_t)m * nl));
    CUDA_TRY(dalloc(&pr->aaS, nl));
    CUDA_TRY(dalloc(&pr->aaRt, (size_t)m * LE));
    CUDA_TRY(dalloc(&pr->aaGt, (size_t)m * LE));
    CUDA_TRY(dalloc(&pr->aaSt, LE));
    CUDA_TRY(dalloc(&pr->aaPt, LE));
    CUDA_TRY(dalloc(&pr->aaP, (size_t)4 * pr->num_sms * kAaDots));
    pr->aa_alloc = m;
    return CCX_OK;
}

bool graph_stale(const ccx_problem* pr, int chunk) {
    return !pr->graph || pr->graph_chunk != chunk || pr->graph_stream != pr->stream_edges ||
           pr->graph_variant != pr->variant || pr->graph_G != pr->G || pr->graph_delta != pr->delta_fuse ||
           pr->graph_aa != pr->aa_use;
}

ccx_status build_graph(ccx_problem* pr, int chunk) {
    if (!graph_stale(pr, chunk)) return CCX_OK;
    if (pr->graph) {
        cudaGraphExecDestroy(pr->graph);
        pr->graph = nullptr;
    }
    // one launch outside capture sets the kernels' shared-memory attributes
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(pr->work, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < chunk && err == cudaSuccess; ++k) {
        if (pr->precision == CCX_FP64) {
            err = launch_pd_iteration_variant<double>(make_params<double>(pr), pr->variant, pr->work);
            if (err == cudaSuccess) err = launch_pd_aa<double>(make_params<double>(pr), pr->work);
        } else {
            err = launch_pd_iteration_variant<float>(make_params<float>(pr), pr->variant, pr->work);
            if (err == cudaSuccess) err = launch_pd_aa<float>(make_params<float>(pr), pr->work);
        }
    }
    cudaError_t e2 = cudaStreamEndCapture(pr->work, &g);
    const unsigned long long kpi = pr->aa_use > 0 ? 4ULL : 2ULL;     // kernels per iteration
    g_launches.fetch_sub(kpi * (unsigned long long)chunk, std::memory_order_relaxed);  // captured, not launched
    if (err != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(CCX_ECUDA, "capturing the iteration graph failed: %s",
                    cudaGetErrorString(err != cudaSuccess ? err : e2));
    }
    err = cudaGraphInstantiate(&pr->graph, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) return fail(CCX_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(err));
    pr->graph_chunk = chunk;
    pr->graph_stream = pr->stream_edges;
    pr->graph_variant = pr->variant;
    pr->graph_G = pr->G;
    pr->graph_delta = pr->delta_fuse;
    pr->graph_aa = pr->aa_use;
    return CCX_OK;
}

// One problem's warm-started path as a resumable sequence of steps, so that one
// host thread can drive one problem (ccx_solve_path, blocking) or several on
// their own streams (ccx_solve_batch, polling).  Per gamma: begin, chunks of
// iterations with one chunk kept queued ahead of the host's check of the state
// word, then the outputs (U, labels) and, once they have landed, the stats.
struct PathRun {
    ccx_problem* pr = nullptr;
    const double* gammas = nullptr;
    int n_gamma = 0;
    ccx_opts o{};
    float* U_out = nullptr;
    int32_t* labels_out = nullptr;
    uint8_t* fused_out = nullptr;  // n_gamma x m fused flags, or NULL
    ccx_gamma_stats* stats = nullptr;
    int pc_q = 0;                  // > 0: write the scores on the principal axes instead of U
    float* scores_out = nullptr;
    bool u_dev = false, l_dev = false, s_dev = false, f_dev = false;
    enum Phase { kIterate, kOutputs, kDone } phase = kDone;
    int g = 0, launched = 0, checked = 0;
    double rho = 0.0, eps = 0.0;
    int conv_hist[3] = {0, 0, 0};  // converged flags of the last three gammas (newest first)
    PdState final{};
    std::chrono::steady_clock::time_point t0;
    bool all_conv = true;
};

template <typename R>
ccx_status path_begin_gamma(PathRun& r) {
    ccx_problem* pr = r.pr;
    const double gamma = r.gammas[r.g];
    r.rho = r.o.rho_scale * (pr->nyc + gamma * pr->nw);
    if (!(r.rho > 0.0)) r.rho = r.o.rho_scale;
    r.eps = (r.o.eps_rel * pr->nyc) * (r.o.eps_rel * pr->nyc);
    if (!(r.eps > 0.0)) r.eps = r.o.eps_rel * r.o.eps_rel;
    const double unit = std::is_same<R, double>::value ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
    const double scale_floor = 64.0 * unit * pr->ny0;
    r.t0 = std::chrono::steady_clock::now();
    if (r.o.extrapolate && r.g >= 1) {
        // predictor along the path in log gamma: on the second gamma A is only
        // recorded; then a secant step (c = spacing ratio, at most 1); with
        // extrapolate = 2, from the fourth gamma on, the quadratic through the
        // last three solutions
        double w0 = 1.0, w1 = 0.0, w2 = 0.0;
        const bool quad = r.o.extrapolate >= 2;
        if (quad && !pr->Aprev2) {
            const size_t nl = (size_t)pr->n * pr->ld;
            const size_t es = std::is_same<R, double>::value ? 8 : 4;
            CUDA_TRY(cudaMalloc(&pr->Aprev2, es * nl));
            if (!std::is_same<R, double>::value) CUDA_TRY(dalloc(&pr->Aprev2_lo, nl));
        }
        auto lg = [&](int k) { return std::log(k == r.g ? gamma : r.gammas[k]); };
        bool pos = gamma > 0.0;
        for (int k = std::max(0, r.g - 3); k < r.g; ++k) pos = pos && r.gammas[k] > 0.0;
        // the quadratic only while the last three gammas stopped on the tolerance: at
        // the rounding floor the solutions differ by noise, which its weights amplify
        const bool smooth = r.conv_hist[0] == 1 && r.conv_hist[1] == 1 && r.conv_hist[2] == 1;
        if (pos && quad && smooth && r.g >= 3) {
            const double x0 = lg(r.g - 3), x1 = lg(r.g - 2), x2 = lg(r.g - 1), x = lg(r.g);
            if (x0 != x1 && x1 != x2 && x0 != x2 && (x - x2) <= (x2 - x1) * 1.0000001) {
                w0 = (x - x1) * (x - x0) / ((x2 - x1) * (x2 - x0));   // weight of A_k
                w1 = (x - x2) * (x - x0) / ((x1 - x2) * (x1 - x0));   // A_(k-1)
                w2 = (x - x2) * (x - x1) / ((x0 - x2) * (x0 - x1));   // A_(k-2)
            }
        } else if (pos && r.g >= 2) {
            const double x1 = lg(r.g - 2), x2 = lg(r.g - 1), x = lg(r.g);
            if (x2 != x1) {
                double c = (x - x2) / (x2 - x1);
                if (!(c > 0.0)) c = 0.0;
                c = std::min(c, 1.0);
                w0 = 1.0 + c;
                w1 = -c;
            }
        }
        CUDA_TRY(launch_pd_extrapolate<R>(make_params<R>(pr), reinterpret_cast<R*>(pr->Aprev), pr->Aprev_lo,
                                          quad ? reinterpret_cast<R*>(pr->Aprev2) : nullptr,
                                          quad ? pr->Aprev2_lo : nullptr, w0, w1, w2, pr->work));
    }
    // the mixing phase only while the path has not started fusing: at a fusion
    // transition the map is not smooth and the restart rule does better
    const int aa_m = (r.o.anderson > 0 && pr->last_fused <= 0) ? r.o.anderson : 0;
    CUDA_TRY(launch_pd_begin_gamma<R>(make_params<R>(pr), gamma, r.rho, r.eps, r.o.tol, r.o.max_iter,
                                      r.o.accelerate, scale_floor, aa_m, pr->work));
    r.launched = r.checked = 0;
    r.phase = PathRun::kIterate;
    return CCX_OK;
}

// Set-up before the first gamma (stream ordering, buffers, first iterate, graph).
template <typename R>
ccx_status path_open(PathRun& r) {
    ccx_problem* pr = r.pr;
    ccx_status s = check_limits(pr);
    if (s != CCX_OK) return s;
    s = enter(pr);
    if (s != CCX_OK) return s;
    s = ensure_path(pr);
    if (s != CCX_OK) return s;
    s = ensure_aa(pr);
    if (s != CCX_OK) return s;
    IterParams<R> P = make_params<R>(pr);
    if (!pr->path_started) {
        const R* Y0 = std::is_same<R, double>::value ? reinterpret_cast<const R*>(pr->Y0d)
                                                      : reinterpret_cast<const R*>(pr->Y0f);
        CUDA_TRY(launch_pd_init<R>(P, Y0, pr->work));
        pr->path_started = true;
    }
    // The first launch of each kernel variant raises its shared-memory limit,
    // which must not happen under capture: launch once on a finished state
    // (done = 1, so every kernel returns at once) before capturing.
    if (graph_stale(pr, r.o.chunk)) CUDA_TRY(launch_pd_iteration_variant<R>(P, pr->variant, pr->work));
    s = build_graph(pr, r.o.chunk);
    if (s != CCX_OK) return s;
    r.u_dev = is_device_ptr(r.U_out);
    r.l_dev = is_device_ptr(r.labels_out);
    r.s_dev = is_device_ptr(r.scores_out);
    r.f_dev = is_device_ptr(r.fused_out);
    r.g = 0;
    r.all_conv = true;
    r.conv_hist[0] = r.conv_hist[1] = r.conv_hist[2] = 0;
    r.phase = PathRun::kDone;
    if (r.n_gamma > 0) return path_begin_gamma<R>(r);
    return CCX_OK;
}

// Advance the run as far as the GPU allows.  With block = false nothing waits:
// *progressed says whether anything happened.  Returns an error status, or OK
// (the run is finished when r.phase == kDone).
template <typename R>
ccx_status path_step(PathRun& r, bool block, bool* progressed) {
    ccx_problem* pr = r.pr;
    *progressed = false;
    if (r.phase == PathRun::kIterate) {
        while (r.launched - r.checked < 2) {
            CUDA_TRY(cudaGraphLaunch(pr->graph, pr->work));
            count_launches((pr->graph_aa > 0 ? 4ULL : 2ULL) * (unsigned long long)pr->graph_chunk);
            CUDA_TRY(cudaMemcpyAsync(&pr->st_host[r.launched & 1], pr->st, sizeof(PdState), cudaMemcpyDeviceToHost,
                                     pr->work));
            CUDA_TRY(cudaEventRecord(pr->ev_chunk[r.launched & 1], pr->work));
            ++r.launched;
            *progressed = true;
        }
        cudaEvent_t ev = pr->ev_chunk[r.checked & 1];
        if (block) {
            CUDA_TRY(cudaEventSynchronize(ev));
        } else {
            const cudaError_t q = cudaEventQuery(ev);
            if (q == cudaErrorNotReady) return CCX_OK;
            CUDA_TRY(q);
        }
        r.final = pr->st_host[r.checked & 1];
        ++r.checked;
        *progressed = true;
        if (!r.final.done) return CCX_OK;
        // The chunk queued behind the finished one returns at once; everything
        // below is ordered after it on the work stream.
        if (r.final.converged == 0) r.all_conv = false;
        pr->last_fused = r.final.n_fused;
        r.conv_hist[2] = r.conv_hist[1];
        r.conv_hist[1] = r.conv_hist[0];
        r.conv_hist[0] = r.final.converged;
        IterParams<R> P = make_params<R>(pr);
        const int g = r.g;
        if (r.U_out) {
            float* dst = r.U_out + (size_t)g * pr->n * pr->ld_in;
            if (r.u_dev) {
                CUDA_TRY(launch_pd_finalize<R>(P, dst, pr->ld_in, (int)pr->p, pr->work));
            } else {
                CUDA_TRY(launch_pd_finalize<R>(P, pr->Ustage, pr->p, (int)pr->p, pr->work));
                CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(float) * pr->ld_in, pr->Ustage, sizeof(float) * pr->p,
                                           sizeof(float) * pr->p, pr->n, cudaMemcpyDeviceToHost, pr->work));
            }
        }
        if (r.pc_q > 0 && r.scores_out) {
            // project on the GPU: only n x q scores leave the device
            CUDA_TRY(launch_pd_finalize<R>(P, pr->Ustage, pr->p, (int)pr->p, pr->work));
            const size_t nq = (size_t)pr->n * r.pc_q;
            float* sdst = r.s_dev ? r.scores_out + (size_t)g * nq : pr->Sstage;
            CUDA_TRY(pc_project(pr->Ustage, (int)pr->p, pr->colmean, pr->pc_axes, (int)pr->n, (int)pr->p, r.pc_q,
                                sdst, pr->work));
            if (!r.s_dev)
                CUDA_TRY(cudaMemcpyAsync(r.scores_out + (size_t)g * nq, pr->Sstage, sizeof(float) * nq,
                                         cudaMemcpyDeviceToHost, pr->work));
        }
        int* ldst = (r.labels_out && r.l_dev) ? r.labels_out + (size_t)g * pr->n : pr->Lstage;
        CUDA_TRY(launch_fused_labels((int)pr->n, P.m, pr->d_ei, pr->d_ej, pr->fused, ldst, pr->d_ncl,
                                     pr->cc_scratch, pr->work));
        if (r.labels_out && !r.l_dev)
            CUDA_TRY(cudaMemcpyAsync(r.labels_out + (size_t)g * pr->n, pr->Lstage, sizeof(int) * pr->n,
                                     cudaMemcpyDeviceToHost, pr->work));
        if (r.fused_out && P.m > 0)
            CUDA_TRY(cudaMemcpyAsync(r.fused_out + (size_t)g * P.m, pr->fused, (size_t)P.m,
                                     r.f_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, pr->work));
        CUDA_TRY(cudaMemcpyAsync(pr->h_ncl, pr->d_ncl, sizeof(int), cudaMemcpyDeviceToHost, pr->work));
        CUDA_TRY(cudaEventRecord(pr->ev_out, pr->work));
        r.phase = PathRun::kOutputs;
    }
    if (r.phase == PathRun::kOutputs) {
        if (block) {
            CUDA_TRY(cudaEventSynchronize(pr->ev_out));
        } else {
            const cudaError_t q = cudaEventQuery(pr->ev_out);
            if (q == cudaErrorNotReady) return CCX_OK;
            CUDA_TRY(q);
        }
        *progressed = true;
        if (*pr->h_ncl < 0)
            return fail(CCX_ECUDA, "gamma %d: the connected-components pass over the fused edges did not settle "
                                   "within n + 1 rounds; labels not written", r.g);
        if (r.stats) {
            ccx_gamma_stats& S = r.stats[r.g];
            S.iters = r.final.iter;
            S.converged = r.final.converged;
            S.n_fused = std::max(r.final.n_fused, 0);
            S.n_clusters = *pr->h_ncl;
            S.gamma = r.gammas[r.g];
            S.rho = r.rho;
            S.eps = r.eps;
            S.d_final = r.final.d_last;
            S.err_est = r.final.err_est;
            S.n_recomputed = r.final.n_recomputed;
            S.recomputes = r.final.recompute_total;
            S.mixing_iters = r.final.aa_total;
            S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - r.t0).count();
        }
        ++r.g;
        if (r.g < r.n_gamma) return path_begin_gamma<R>(r);
        r.phase = PathRun::kDone;
    }
    return CCX_OK;
}

ccx_status path_open_any(PathRun& r) {
    return r.pr->precision == CCX_FP64 ? path_open<double>(r) : path_open<float>(r);
}

ccx_status path_step_any(PathRun& r, bool block, bool* progressed) {
    return r.pr->precision == CCX_FP64 ? path_step<double>(r, block, progressed)
                                       : path_step<float>(r, block, progressed);
}

// Final status of a run that reached kDone, after its stream ordering is closed.
ccx_status path_close(PathRun& r, ccx_status run_status) {
    std::string keep = g_err;
    const ccx_status l = leave(r.pr);
    if (run_status != CCX_OK) {
        g_err = keep;
        return run_status;
    }
    if (l != CCX_OK) return l;
    if (!r.all_conv) return fail(CCX_ENOTCONV, "max_iter reached before convergence for some gamma");
    return CCX_OK;
}

// Y_0 (missing entries at observed column means), its column means and the
// norms ||Y_c||_F and ||Y_0||_F that fix rho, eps and the error floor.
ccx_status prepare_start(ccx_problem* pr) {
    const int64_t n = pr->n, p = pr->p;
    CUDA_TRY(launch_fill_missing(pr->Xf, pr->Xd, pr->maskbits, (int)n, (int)p, pr->ld, pr->ldw, pr->colmean,
                                 pr->Y0f, pr->Y0d, pr->d_ss, pr->work));
    double ss = 0.0;
    std::vector<double> cm(p);
    CUDA_TRY(cudaMemcpyAsync(&ss, pr->d_ss, sizeof(double), cudaMemcpyDeviceToHost, pr->work));
    CUDA_TRY(cudaMemcpyAsync(cm.data(), pr->colmean, sizeof(double) * p, cudaMemcpyDeviceToHost, pr->work));
    CUDA_TRY(cudaStreamSynchronize(pr->work));
    pr->nyc = std::sqrt(ss);
    double s0 = 0.0;
    for (int64_t c = 0; c < p; ++c) s0 += cm[c] * cm[c];
    pr->ny0 = std::sqrt(ss + (double)n * s0);   // ||Y_0||^2 = ||Y_c||^2 + n ||mean||^2
    return CCX_OK;
}

// Options of one solve, validated; the FP64 default tolerance is tighter.
ccx_status resolve_opts(const ccx_problem* pr, const ccx_opts* opts, ccx_opts* o) {
    ccx_opts_default(o);
    if (pr->precision == CCX_FP64) o->tol = 1e-10;
    if (opts) *o = *opts;
    if (!(o->rho_scale > 0.0) || !std::isfinite(o->rho_scale)) return fail(CCX_EINVAL, "rho_scale must be > 0");
    if (!(o->eps_rel > 0.0) || !std::isfinite(o->eps_rel)) return fail(CCX_EINVAL, "eps_rel must be > 0");
    if (!(o->tol > 0.0)) return fail(CCX_EINVAL, "tol must be > 0");
    if (o->max_iter < 1) return fail(CCX_EINVAL, "max_iter must be >= 1");
    if (o->chunk < 1 || o->chunk > 4096) return fail(CCX_EINVAL, "chunk must be in [1, 4096]");
    if (o->slice_variant < 0 || o->slice_variant > 2) return fail(CCX_EINVAL, "slice_variant must be 0, 1 or 2");
    if (o->max_ctas < 0) return fail(CCX_EINVAL, "max_ctas must be >= 0");
    if (!(o->fuse_delta >= 0.0 && o->fuse_delta < 1.0)) return fail(CCX_EINVAL, "fuse_delta must be in [0, 1)");
    if (o->anderson < 0 || o->anderson > kAaMax) return fail(CCX_EINVAL, "anderson must be in [0, %d]", kAaMax);
    return CCX_OK;
}

ccx_status check_gammas(const double* gammas, int n_gamma) {
    if (n_gamma < 0) return fail(CCX_EINVAL, "n_gamma < 0");
    if (n_gamma > 0 && !gammas) return fail(CCX_EINVAL, "gammas is NULL");
    for (int g = 0; g < n_gamma; ++g)
        if (!std::isfinite(gammas[g]) || gammas[g] < 0.0)
            return fail(CCX_EINVAL, "gammas[%d] must be finite and >= 0", g);
    return CCX_OK;
}

}  // namespace

extern "C" {

void ccx_opts_default(ccx_opts* o) {
    if (!o) return;
    o->rho_scale = 2.0;
    o->eps_rel = 1e-3;
    o->tol = 1e-6;
    o->max_iter = 200000;
    o->accelerate = 1;
    o->chunk = 64;
    o->extrapolate = 1;
    o->stream_edges = 0;
    o->slice_variant = 0;
    o->max_ctas = 0;
    o->fuse_delta = 1e-5;
    o->anderson = 0;
}

const char* ccx_last_error(void) { return g_err.c_str(); }

const char* ccx_version(void) { return "ccx 0.1 (sm_103a)"; }

ccx_status ccx_problem_create(const float* X, const uint8_t* mask, int64_t n, int64_t p, int64_t ld, int precision,
                              void* stream, ccx_problem** out) {
    g_err.clear();
    if (!out) return fail(CCX_EINVAL, "out is NULL");
    *out = nullptr;
    if (!X) return fail(CCX_EINVAL, "X is NULL");
    if (n < 1 || p < 1) return fail(CCX_EINVAL, "need n >= 1 and p >= 1 (got %lld, %lld)", (long long)n, (long long)p);
    if (ld < p) return fail(CCX_EINVAL, "ld (%lld) < p (%lld)", (long long)ld, (long long)p);
    if (precision != CCX_FP32 && precision != CCX_FP64) return fail(CCX_EINVAL, "precision must be CCX_FP32 or CCX_FP64");
    if (n > (int64_t)1 << 30 || p > (int64_t)1 << 30) return fail(CCX_EINVAL, "n or p too large");
    ccx_problem* pr = new ccx_problem();
    pr->precision = precision;
    pr->n = n;
    pr->p = p;
    pr->ld_in = ld;
    pr->ld = (int)((p + 31) / 32 * 32);
    pr->ldw = pr->ld / 32;
    pr->has_mask = mask != nullptr;
    pr->user = reinterpret_cast<cudaStream_t>(stream);
    auto bail = [&](ccx_status s) {
        free_all(pr);
        delete pr;
        return s;
    };
#define TRY(expr)                                                                                  \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess)                                                                     \
            return bail(fail(_e == cudaErrorMemoryAllocation ? CCX_ENOMEM : CCX_ECUDA, "%s: %s", #expr, \
                             cudaGetErrorString(_e)));                                             \
    } while (0)
    TRY(cudaGetDevice(&pr->device));
    TRY(cudaDeviceGetAttribute(&pr->num_sms, cudaDevAttrMultiProcessorCount, pr->device));
    TRY(cudaStreamCreateWithFlags(&pr->work, cudaStreamNonBlocking));
    TRY(cudaEventCreateWithFlags(&pr->ev_user, cudaEventDisableTiming));
    TRY(cudaEventCreateWithFlags(&pr->ev_done, cudaEventDisableTiming));
    TRY(cudaEventCreateWithFlags(&pr->ev_chunk[0], cudaEventDisableTiming));
    TRY(cudaEventCreateWithFlags(&pr->ev_chunk[1], cudaEventDisableTiming));
    TRY(cudaEventCreateWithFlags(&pr->ev_out, cudaEventDisableTiming));
    TRY(cudaEventRecord(pr->ev_user, pr->user));
    TRY(cudaStreamWaitEvent(pr->work, pr->ev_user, 0));
    const size_t nl = (size_t)n * pr->ld;
    TRY(dalloc(&pr->Xf, nl));
    if (precision == CCX_FP64) TRY(dalloc(&pr->Xd, nl));
    if (mask) TRY(dalloc(&pr->maskbits, (size_t)n * pr->ldw));
    TRY(dalloc(&pr->colmean, 2 * (size_t)pr->ld));
    TRY(dalloc(&pr->Y0f, nl));
    if (precision == CCX_FP64) TRY(dalloc(&pr->Y0d, nl));
    TRY(dalloc(&pr->d_ss, 1));
    // stage caller arrays on the device
    const float* Xsrc = X;
    const uint8_t* Msrc = mask;
    float* Xtmp = nullptr;
    uint8_t* Mtmp = nullptr;
    int* bad = nullptr;
    if (!is_device_ptr(X)) {
        TRY(dalloc(&Xtmp, (size_t)n * ld));
        TRY(cudaMemcpyAsync(Xtmp, X, sizeof(float) * (size_t)n * ld, cudaMemcpyHostToDevice, pr->work));
        Xsrc = Xtmp;
    }
    if (mask && !is_device_ptr(mask)) {
        TRY(dalloc(&Mtmp, (size_t)n * ld));
        TRY(cudaMemcpyAsync(Mtmp, mask, (size_t)n * ld, cudaMemcpyHostToDevice, pr->work));
        Msrc = Mtmp;
    }
    TRY(dalloc(&bad, 2));
    TRY(cudaMemsetAsync(bad, 0, 2 * sizeof(int), pr->work));
    TRY(launch_pack_input(Xsrc, Msrc, n, p, ld, pr->Xf, pr->Xd, pr->maskbits, pr->ld, pr->ldw, bad, pr->work));
    int hbad[2] = {0, 0};
    TRY(cudaMemcpyAsync(hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, pr->work));
    TRY(cudaStreamSynchronize(pr->work));
    cudaFree(Xtmp);
    cudaFree(Mtmp);
    cudaFree(bad);
    if (hbad[0] > 0) return bail(fail(CCX_EINVAL, "%d observed entries of X are not finite", hbad[0]));
    if (hbad[1] > 0) return bail(fail(CCX_EINVAL, "%d rows have no observed entry", hbad[1]));
    {
        const ccx_status st = prepare_start(pr);
        if (st != CCX_OK) return bail(st);
    }
    // an empty edge set until the caller sets or builds one
    {
        std::vector<int> e0;
        std::vector<double> w0;
        ccx_status s = install_edges(pr, e0, e0, w0);
        if (s != CCX_OK) return bail(s);
    }
#undef TRY
    *out = pr;
    return CCX_OK;
}

ccx_status ccx_standardize(ccx_problem* pr) {
    g_err.clear();
    if (!pr) return fail(CCX_EINVAL, "problem is NULL");
    ccx_status s = enter(pr);
    if (s != CCX_OK) return s;
    CUDA_TRY(launch_standardize(pr->Xf, pr->Xd, pr->has_mask ? pr->maskbits : nullptr, (int)pr->n, (int)pr->p, pr->ld,
                                pr->ldw, pr->colmean, pr->work));
    s = prepare_start(pr);
    if (s != CCX_OK) return s;
    // the data changed: weights, principal axes and the path state no longer apply
    cudaFree(pr->pc_axes);
    cudaFree(pr->Sstage);
    pr->pc_axes = nullptr;
    pr->Sstage = nullptr;
    pr->pc_q = 0;
    std::vector<int> e0;
    std::vector<double> w0;
    s = install_edges(pr, e0, e0, w0);
    if (s != CCX_OK) return s;
    drop_shard(pr);
    return leave(pr);
}

ccx_status ccx_get_start(const ccx_problem* pr_c, float* Y0_out) {
    g_err.clear();
    ccx_problem* pr = const_cast<ccx_problem*>(pr_c);
    if (!pr || !Y0_out) return fail(CCX_EINVAL, "NULL argument");
    ccx_status s = enter(pr);
    if (s != CCX_OK) return s;
    CUDA_TRY(cudaMemcpy2DAsync(Y0_out, sizeof(float) * pr->p, pr->Y0f, sizeof(float) * pr->ld, sizeof(float) * pr->p,
                               pr->n, is_device_ptr(Y0_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               pr->work));
    return leave(pr);
}

ccx_status ccx_set_edges(ccx_problem* pr, int64_t n_edges, const int32_t* ei, const int32_t* ej, const double* w) {
    g_err.clear();
    if (!pr) return fail(CCX_EINVAL, "problem is NULL");
    if (n_edges < 0) return fail(CCX_EINVAL, "n_edges < 0");
    if (n_edges > 0 && (!ei || !ej || !w)) return fail(CCX_EINVAL, "edge arrays are NULL");
    CUDA_TRY(cudaSetDevice(pr->device));
    std::vector<int> a(ei, ei + n_edges), b(ej, ej + n_edges);
    std::vector<double> c(w, w + n_edges);
    return install_edges(pr, a, b, c);
}

ccx_status ccx_build_knn(ccx_problem* pr, const ccx_knn_rule* rule) {
    g_err.clear();
    if (!pr || !rule) return fail(CCX_EINVAL, "NULL argument");
    if (rule->k < 1) return fail(CCX_EINVAL, "k must be >= 1");
    if (!rule->phi_auto && (!std::isfinite(rule->phi) || rule->phi < 0.0))
        return fail(CCX_EINVAL, "phi must be finite and >= 0");
    if (rule->gram < 0 || rule->gram > 2) return fail(CCX_EINVAL, "gram must be 0, 1 or 2");
    ccx_status s = enter(pr);
    if (s != CCX_OK) return s;
    knn_set_exact_rows(pr->Xf, pr->has_mask ? pr->maskbits : nullptr, pr->colmean, pr->ldw);
    KnnResult res;
    std::string err;
    cudaError_t e = knn_build(pr->Y0f, (int)pr->n, (int)pr->p, pr->ld, rule->k, rule->phi, rule->phi_auto,
                              rule->normalize, pr->work, &res, &err, nullptr, 1.0, 0, rule->gram);
    if (e == cudaErrorNotSupported) return fail(CCX_EUNSUPPORTED, "%s", err.c_str());
    if (e != cudaSuccess) return fail(CCX_ECUDA, "kNN build failed: %s", cudaGetErrorString(e));
    s = install_edges(pr, res.ei, res.ej, res.w);
    if (s != CCX_OK) return s;
    return leave(pr);
}

ccx_status ccx_build_knn_composite(ccx_problem* pr, const ccx_knn_rule* rule, const double* coords, double alpha,
                                   int geodesic) {
    g_err.clear();
    if (!pr || !rule || !coords) return fail(CCX_EINVAL, "NULL argument");
    if (rule->k < 1) return fail(CCX_EINVAL, "k must be >= 1");
    if (!rule->phi_auto && (!std::isfinite(rule->phi) || rule->phi < 0.0))
        return fail(CCX_EINVAL, "phi must be finite and >= 0");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(CCX_EINVAL, "alpha must be in [0, 1]");
    if (rule->gram < 0 || rule->gram > 2) return fail(CCX_EINVAL, "gram must be 0, 1 or 2");
    for (int64_t i = 0; i < pr->n; ++i) {
        const double la = coords[2 * i], lo = coords[2 * i + 1];
        if (!std::isfinite(la) || !std::isfinite(lo) || la < -90.0 || la > 90.0)
            return fail(CCX_EINVAL, "coords[%lld]: latitude must be in [-90, 90] and both finite", (long long)i);
    }
    ccx_status s = enter(pr);
    if (s != CCX_OK) return s;
    double* geo = nullptr;
    CUDA_TRY(dalloc(&geo, 2 * (size_t)pr->n));
    cudaError_t e = cudaMemcpyAsync(geo, coords, sizeof(double) * 2 * pr->n, cudaMemcpyHostToDevice, pr->work);
    knn_set_exact_rows(pr->Xf, pr->has_mask ? pr->maskbits : nullptr, pr->colmean, pr->ldw);
    KnnResult res;
    std::string err;
    if (e == cudaSuccess)
        e = knn_build(pr->Y0f, (int)pr->n, (int)pr->p, pr->ld, rule->k, rule->phi, rule->phi_auto, rule->normalize,
                      pr->work, &res, &err, geo, alpha, geodesic ? 1 : 0, rule->gram);
    cudaFree(geo);
    if (e == cudaErrorNotSupported) return fail(CCX_EUNSUPPORTED, "%s", err.c_str());
    if (e != cudaSuccess) return fail(CCX_ECUDA, "kNN build failed: %s", cudaGetErrorString(e));
    s = install_edges(pr, res.ei, res.ej, res.w);
    if (s != CCX_OK) return s;
    return leave(pr);
}

ccx_status ccx_sweep_plan(int64_t n, int64_t n_edges, const int32_t* ei, const int32_t* ej, int precision,
                          int32_t* sizes, int32_t* node_row, int32_t* node_nbr, int32_t* edge_id) {
    g_err.clear();
    if (!sizes) return fail(CCX_EINVAL, "sizes is NULL");
    if (n < 1 || n > 65535) return fail(CCX_EINVAL, "n must be in [1, 65535]");
    if (n_edges < 0 || n_edges > (int64_t)1 << 30) return fail(CCX_EINVAL, "bad n_edges");
    if (n_edges > 0 && (!ei || !ej)) return fail(CCX_EINVAL, "ei or ej is NULL");
    if (precision != CCX_FP32 && precision != CCX_FP64) return fail(CCX_EINVAL, "precision must be 0 or 1");
    std::vector<int> a(n_edges), b(n_edges);
    for (int64_t q = 0; q < n_edges; ++q) {
        a[q] = ei[q];
        b[q] = ej[q];
        if (a[q] < 0 || b[q] >= n || a[q] >= b[q])
            return fail(CCX_EINVAL, "edge %lld: need 0 <= ei < ej < n", (long long)q);
        if (q > 0 && (a[q] < a[q - 1] || (a[q] == a[q - 1] && b[q] <= b[q - 1])))
            return fail(CCX_EINVAL, "edges must be sorted by (ei, ej) without duplicates");
    }
    const SweepPlan P = plan_sweeps(n, a, b, precision);
    const int T = kSliceThreads;
    sizes[0] = T;
    sizes[1] = P.la;
    sizes[2] = P.le;
    sizes[3] = P.nslots;
    const size_t LA = (size_t)P.la * T, LE = (size_t)P.le * T;
    for (size_t x = 0; x < LA; ++x) {
        if (node_row) node_row[x] = P.node_row[x];
        if (node_nbr) node_nbr[x] = P.node_row[x] >= 0 ? (int32_t)P.csrT[x] : -1;
    }
    if (edge_id)
        for (size_t x = 0; x < LE; ++x) edge_id[x] = P.eid[x];
    return CCX_OK;
}

ccx_status ccx_min_connected_k(ccx_problem* pr, int k_max, int* k_out) {
    g_err.clear();
    if (!pr || !k_out) return fail(CCX_EINVAL, "NULL argument");
    if (k_max < 1) return fail(CCX_EINVAL, "k_max must be >= 1");
    if (pr->n < 2) return fail(CCX_EINVAL, "need at least two cases");
    ccx_status s = enter(pr);
    if (s != CCX_OK) return s;
    knn_set_exact_rows(pr->Xf, pr->has_mask ? pr->maskbits : nullptr, pr->colmean, pr->ldw);
    std::string err;
    int probes = 0;
    const cudaError_t e =
        knn_min_connected_k(pr->Y0f, (int)pr->n, (int)pr->p, pr->ld, k_max, pr->work, k_out, &probes, &err);
    if (e == cudaErrorNotSupported) return fail(CCX_EUNSUPPORTED, "%s", err.c_str());
    if (e != cudaSuccess) return fail(CCX_ECUDA, "connectivity search failed: %s", cudaGetErrorString(e));
    return leave(pr);
}

ccx_status ccx_get_edges(const ccx_problem* pr, int64_t* n_edges, int32_t* ei, int32_t* ej, double* w) {
    g_err.clear();
    if (!pr || !n_edges) return fail(CCX_EINVAL, "NULL argument");
    const int64_t m = (int64_t)pr->ei.size();
    if (!ei) {
        *n_edges = m;
        return CCX_OK;
    }
    if (*n_edges < m) return fail(CCX_EINVAL, "capacity %lld < %lld edges", (long long)*n_edges, (long long)m);
    std::copy(pr->ei.begin(), pr->ei.end(), ei);
    if (ej) std::copy(pr->ej.begin(), pr->ej.end(), ej);
    if (w) std::copy(pr->w.begin(), pr->w.end(), w);
    *n_edges = m;
    return CCX_OK;
}

ccx_status ccx_fusion_scale(const ccx_problem* pr_c, double* gamma0) {
    g_err.clear();
    ccx_problem* pr = const_cast<ccx_problem*>(pr_c);
    if (!pr || !gamma0) return fail(CCX_EINVAL, "NULL argument");
    const int m = (int)pr->ei.size();
    if (m == 0) return fail(CCX_EINVAL, "no edges");
    ccx_status s = enter(pr);
    if (s != CCX_OK) return s;
    double* d2 = nullptr;
    CUDA_TRY(dalloc(&d2, m));
    cudaError_t e = edge_distances(pr->Y0f, (int)pr->n, (int)pr->p, pr->ld, pr->d_ei, pr->d_ej, m, d2, pr->work);
    std::vector<double> h(m);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d2, sizeof(double) * m, cudaMemcpyDeviceToHost, pr->work);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pr->work);
    cudaFree(d2);
    if (e != cudaSuccess) return fail(CCX_ECUDA, "fusion scale: %s", cudaGetErrorString(e));
    for (int q = 0; q < m; ++q) h[q] = std::sqrt(h[q]) / (2.0 * pr->w[q]);
    std::sort(h.begin(), h.end());
    *gamma0 = (m % 2) ? h[m / 2] : 0.5 * (h[m / 2 - 1] + h[m / 2]);
    return leave(pr);
}

namespace {
// host copy of the per-edge ratios for the allocation-free variant below
double g_ratio_host[kStaticEdgesMax];
std::mutex g_ratio_mu;
}  // namespace

ccx_status ccx_fusion_scale_noalloc(const ccx_problem* pr_c, double* gamma0) {
    g_err.clear();
    ccx_problem* pr = const_cast<ccx_problem*>(pr_c);
    if (!pr || !gamma0) return fail(CCX_EINVAL, "NULL argument");
    const int64_t m = (int64_t)pr->ei.size();
    if (m == 0) return fail(CCX_EINVAL, "no edges");
    if (m > kStaticEdgesMax)
        return fail(CCX_EINVAL, "ccx_fusion_scale_noalloc handles at most %d edges, this problem has %lld; "
                                "use ccx_fusion_scale", kStaticEdgesMax, (long long)m);
    std::lock_guard<std::mutex> lk(g_ratio_mu);
    ccx_status s = enter(pr);
    if (s != CCX_OK) return s;
    double* scratch = nullptr;
    CUDA_TRY(static_edge_scratch(&scratch));
    CUDA_TRY(edge_ratios_static(pr->Y0f, (int)pr->p, pr->ld, pr->d_ei, pr->d_ej, pr->d_w, (int)m, scratch, pr->work));
    CUDA_TRY(cudaMemcpyAsync(g_ratio_host, scratch, sizeof(double) * m, cudaMemcpyDeviceToHost, pr->work));
    s = leave(pr);
    if (s != CCX_OK) return s;
    // median without a sort buffer: the upper middle by selection, the lower
    // middle (even m) as the largest element left of it
    double* h = g_ratio_host;
    std::nth_element(h, h + m / 2, h + m);
    const double hi = h[m / 2];
    *gamma0 = (m % 2) ? hi : 0.5 * (*std::max_element(h, h + m / 2) + hi);
    return CCX_OK;
}

ccx_status ccx_solve_path(ccx_problem* pr, const double* gammas, int n_gamma, const ccx_opts* opts, float* U_out,
                          int32_t* labels_out, ccx_gamma_stats* stats) {
    return ccx_solve_path_fused(pr, gammas, n_gamma, opts, U_out, labels_out, nullptr, stats);
}

ccx_status ccx_solve_path_fused(ccx_problem* pr, const double* gammas, int n_gamma, const ccx_opts* opts,
                                float* U_out, int32_t* labels_out, uint8_t* fused_out, ccx_gamma_stats* stats) {
    g_err.clear();
    if (!pr) return fail(CCX_EINVAL, "problem is NULL");
    ccx_status s = check_gammas(gammas, n_gamma);
    if (s != CCX_OK) return s;
    PathRun r;
    s = resolve_opts(pr, opts, &r.o);
    if (s != CCX_OK) return s;
    apply_opts(pr, r.o);
    r.pr = pr;
    r.gammas = gammas;
    r.n_gamma = n_gamma;
    r.U_out = U_out;
    r.labels_out = labels_out;
    r.fused_out = fused_out;
    r.stats = stats;
    s = path_open_any(r);
    if (s != CCX_OK) return s;
    while (s == CCX_OK && r.phase != PathRun::kDone) {
        bool progressed = false;
        s = path_step_any(r, true, &progressed);
    }
    return path_close(r, s);
}

namespace {
// principal axes cached on the problem (recomputed when q changes)
ccx_status ensure_axes(ccx_problem* pr, int q) {
    if (q < 1 || q > pc_max_axes()) return fail(CCX_EINVAL, "q must be in [1, %d]", pc_max_axes());
    if (q > std::min<int64_t>(pr->n, pr->p)) return fail(CCX_EINVAL, "q must be <= min(n, p)");
    if (pr->pc_axes && pr->pc_q == q) return CCX_OK;
    cudaFree(pr->pc_axes);
    cudaFree(pr->Sstage);
    pr->pc_axes = nullptr;
    pr->Sstage = nullptr;
    pr->pc_q = 0;
    CUDA_TRY(dalloc(&pr->pc_axes, (size_t)q * pr->p));
    CUDA_TRY(dalloc(&pr->Sstage, (size_t)q * pr->n));
    pr->pc_var.assign(q, 0.0);
    CUDA_TRY(pc_axes(pr->Y0f, pr->colmean, (int)pr->n, (int)pr->p, pr->ld, q, pr->pc_axes, pr->pc_var.data(),
                     pr->work));
    pr->pc_q = q;
    return CCX_OK;
}
}  // namespace

ccx_status ccx_principal_axes(ccx_problem* pr, int q, double* axes_out, double* var_out) {
    g_err.clear();
    if (!pr) return fail(CCX_EINVAL, "problem is NULL");
    ccx_status s = enter(pr);
    if (s != CCX_OK) return s;
    s = ensure_axes(pr, q);
    if (s != CCX_OK) return s;
    if (axes_out)
        CUDA_TRY(cudaMemcpyAsync(axes_out, pr->pc_axes, sizeof(double) * (size_t)q * pr->p, cudaMemcpyDeviceToHost,
                                 pr->work));
    if (var_out) std::copy(pr->pc_var.begin(), pr->pc_var.end(), var_out);
    return leave(pr);
}

ccx_status ccx_solve_path_projected(ccx_problem* pr, const double* gammas, int n_gamma, const ccx_opts* opts, int q,
                                    float* scores_out, int32_t* labels_out, ccx_gamma_stats* stats) {
    g_err.clear();
    if (!pr) return fail(CCX_EINVAL, "problem is NULL");
    ccx_status s = check_gammas(gammas, n_gamma);
    if (s != CCX_OK) return s;
    PathRun r;
    s = resolve_opts(pr, opts, &r.o);
    if (s != CCX_OK) return s;
    s = enter(pr);
    if (s != CCX_OK) return s;
    s = ensure_axes(pr, q);
    if (s != CCX_OK) return s;
    apply_opts(pr, r.o);
    r.pr = pr;
    r.gammas = gammas;
    r.n_gamma = n_gamma;
    r.pc_q = q;
    r.scores_out = scores_out;
    r.labels_out = labels_out;
    r.stats = stats;
    s = path_open_any(r);
    if (s != CCX_OK) return s;
    while (s == CCX_OK && r.phase != PathRun::kDone) {
        bool progressed = false;
        s = path_step_any(r, true, &progressed);
    }
    return path_close(r, s);
}

ccx_status ccx_solve_batch(ccx_problem* const* probs, int n_probs, const double* const* gammas, const int* n_gamma,
                           const ccx_opts* opts, float* const* U_out, int32_t* const* labels_out,
                           ccx_gamma_stats* const* stats, int max_active, ccx_status* status) {
    g_err.clear();
    if (n_probs < 0) return fail(CCX_EINVAL, "n_probs < 0");
    if (n_probs == 0) return CCX_OK;
    if (!probs || !gammas || !n_gamma) return fail(CCX_EINVAL, "probs, gammas and n_gamma must not be NULL");
    for (int i = 0; i < n_probs; ++i) {
        if (!probs[i]) return fail(CCX_EINVAL, "probs[%d] is NULL", i);
        for (int j = 0; j < i; ++j)
            if (probs[j] == probs[i]) return fail(CCX_EINVAL, "probs[%d] and probs[%d] are the same problem", j, i);
        ccx_status s = check_gammas(gammas[i], n_gamma[i]);
        if (s != CCX_OK) return fail(s, "problem %d: %s", i, g_err.c_str());
    }
    if (max_active <= 0) max_active = 32;
    std::vector<PathRun> runs(n_probs);
    std::vector<ccx_status> st(n_probs, CCX_OK);
    std::vector<std::string> msg(n_probs);
    for (int i = 0; i < n_probs; ++i) {
        PathRun& r = runs[i];
        ccx_status s = resolve_opts(probs[i], opts, &r.o);
        if (s != CCX_OK) return fail(s, "problem %d: %s", i, g_err.c_str());
        r.pr = probs[i];
        r.gammas = gammas[i];
        r.n_gamma = n_gamma[i];
        r.U_out = U_out ? U_out[i] : nullptr;
        r.labels_out = labels_out ? labels_out[i] : nullptr;
        r.stats = stats ? stats[i] : nullptr;
    }
    // Problems run on their own work streams; up to max_active of them have
    // chunks queued at once, so small problems share the GPU.  The host polls
    // without blocking and sleeps briefly when no run moved.
    std::vector<int> active;
    int next = 0, finished = 0;
    auto retire = [&](int i, ccx_status s) {
        st[i] = path_close(runs[i], s);
        if (st[i] != CCX_OK) msg[i] = g_err;
        ++finished;
    };
    while (finished < n_probs) {
        while ((int)active.size() < max_active && next < n_probs) {
            const int i = next++;
            g_err.clear();
            apply_opts(runs[i].pr, runs[i].o);
            const ccx_status s = path_open_any(runs[i]);
            if (s != CCX_OK) {
                st[i] = s;
                msg[i] = g_err;
                ++finished;
                continue;
            }
            if (runs[i].phase == PathRun::kDone) retire(i, CCX_OK);
            else active.push_back(i);
        }
        bool any = false;
        for (size_t a = 0; a < active.size();) {
            const int i = active[a];
            bool progressed = false;
            g_err.clear();
            const ccx_status s = path_step_any(runs[i], false, &progressed);
            any = any || progressed;
            if (s != CCX_OK || runs[i].phase == PathRun::kDone) {
                retire(i, s);
                active.erase(active.begin() + (long)a);
            } else {
                ++a;
            }
        }
        if (!any && !active.empty()) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    ccx_status worst = CCX_OK;
    int first = -1;
    for (int i = 0; i < n_probs; ++i) {
        if (status) status[i] = st[i];
        if (st[i] != CCX_OK && st[i] != CCX_ENOTCONV && first < 0) first = i;
        if (st[i] == CCX_ENOTCONV && worst == CCX_OK) worst = CCX_ENOTCONV;
    }
    if (first >= 0) return fail(st[first], "problem %d: %s", first, msg[first].c_str());
    if (worst == CCX_ENOTCONV) return fail(CCX_ENOTCONV, "max_iter reached before convergence for some gamma");
    return CCX_OK;
}

// ------------------------------------------------------------------ serving
namespace {

// Device bytes ensure_path allocates for a problem's iteration (admission estimate).
size_t path_bytes(const ccx_problem* pr) {
    const bool fp64 = pr->precision == CCX_FP64;
    const size_t es = fp64 ? 8 : 4;
    const size_t nl = (size_t)pr->n * pr->ld;
    const size_t m = pr->ei.size();
    const size_t nsl = (size_t)((pr->p + kSliceCols - 1) / kSliceCols);
    const size_t G = std::min<size_t>(nsl, (size_t)std::max(pr->num_sms, 1));
    const size_t T = kSliceThreads;
    size_t b = 5 * es * nl + (fp64 ? 0 : 3 * 4 * nl) + (pr->has_mask ? 2 * es * nl : 0);
    b += 2 * es * 2 * ((size_t)pr->la + pr->le) * T;
    b += G * (size_t)pr->le * T * 4 + G * 64 + m * 9 + 24 * (size_t)pd_reduce_blocks(pr->le);
    b += (size_t)pr->n * pr->p * 4 + (size_t)pr->n * 8 + 4096;
    return b + b / 16 + (1u << 20);   // allocation rounding
}

}  // namespace

struct ccx_server {
    struct Job {
        uint64_t ticket = 0;
        ccx_problem* pr = nullptr;
        std::vector<double> gammas;
        float* U_out = nullptr;
        int32_t* labels_out = nullptr;
        ccx_gamma_stats* stats = nullptr;
        size_t bytes = 0;
        PathRun run;
        bool done = false;
        ccx_status status = CCX_OK;
        std::string msg;
    };
    ccx_opts opts{};
    size_t budget = 0;
    int max_active = 32;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> pending;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;   // submitted and not yet waited for
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;

    void finish(const std::shared_ptr<Job>& j, ccx_status st, const std::string& m) {
        std::lock_guard<std::mutex> lk(mu);
        j->status = st;
        j->msg = m;
        j->done = true;
        cv_done.notify_all();
    }

    // The scheduler: admits queued jobs while the estimated device memory of
    // the running ones stays within the budget (one job always runs), steps
    // every running job without blocking, and releases a job's iteration
    // buffers when it finishes.
    void loop() {
        cudaSetDevice(device);
        std::vector<std::shared_ptr<Job>> active;
        size_t used = 0;
        for (;;) {
            std::vector<std::shared_ptr<Job>> admitted;
            {
                std::unique_lock<std::mutex> lk(mu);
                if (active.empty() && pending.empty()) {
                    if (stop) break;
                    cv_work.wait(lk, [&] { return stop || !pending.empty(); });
                    continue;
                }
                while (!pending.empty() && (int)active.size() < max_active) {
                    auto& j = pending.front();
                    if (!active.empty() && used + j->bytes > budget) break;
                    used += j->bytes;
                    active.push_back(j);
                    admitted.push_back(j);
                    pending.pop_front();
                }
            }
            for (auto& j : admitted) {
                g_err.clear();
                apply_opts(j->pr, j->run.o);
                const ccx_status st = path_open_any(j->run);
                if (st != CCX_OK || j->run.phase == PathRun::kDone) {
                    const ccx_status fin = st != CCX_OK ? st : path_close(j->run, CCX_OK);
                    const std::string m = g_err;
                    free_path(j->pr);
                    used -= j->bytes;
                    active.erase(std::find(active.begin(), active.end(), j));
                    finish(j, fin, m);
                }
            }
            bool any = false;
            for (size_t a = 0; a < active.size();) {
                auto j = active[a];
                bool progressed = false;
                g_err.clear();
                ccx_status st = path_step_any(j->run, false, &progressed);
                any = any || progressed;
                if (st != CCX_OK || j->run.phase == PathRun::kDone) {
                    st = path_close(j->run, st);
                    const std::string m = g_err;
                    free_path(j->pr);
                    used -= j->bytes;
                    active.erase(active.begin() + (long)a);
                    finish(j, st, m);
                } else {
                    ++a;
                }
            }
            if (!any) {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait_for(lk, std::chrono::microseconds(20));
            }
        }
    }
};

ccx_status ccx_server_create(const ccx_opts* opts, size_t hbm_budget, int max_active, ccx_server** out) {
    g_err.clear();
    if (!out) return fail(CCX_EINVAL, "out is NULL");
    *out = nullptr;
    auto srv = std::make_unique<ccx_server>();
    ccx_opts_default(&srv->opts);
    if (opts) srv->opts = *opts;
    CUDA_TRY(cudaGetDevice(&srv->device));
    if (hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        hbm_budget = fr / 5 * 4;
    }
    srv->budget = hbm_budget;
    srv->max_active = max_active > 0 ? max_active : 32;
    ccx_server* raw = srv.get();
    try {
        srv->worker = std::thread([raw] { raw->loop(); });
    } catch (...) {
        return fail(CCX_ENOMEM, "could not start the server thread");
    }
    *out = srv.release();
    return CCX_OK;
}

ccx_status ccx_submit(ccx_server* srv, ccx_problem* pr, const double* gammas, int n_gamma, float* U_out,
                      int32_t* labels_out, ccx_gamma_stats* stats, uint64_t* ticket) {
    g_err.clear();
    if (!srv || !pr || !ticket) return fail(CCX_EINVAL, "NULL argument");
    ccx_status s = check_gammas(gammas, n_gamma);
    if (s != CCX_OK) return s;
    auto j = std::make_shared<ccx_server::Job>();
    s = resolve_opts(pr, &srv->opts, &j->run.o);
    if (s != CCX_OK) return s;
    j->pr = pr;
    j->gammas.assign(gammas, gammas + n_gamma);
    j->U_out = U_out;
    j->labels_out = labels_out;
    j->stats = stats;
    j->bytes = path_bytes(pr);
    j->run.pr = pr;
    j->run.n_gamma = n_gamma;
    j->run.U_out = U_out;
    j->run.labels_out = labels_out;
    j->run.stats = stats;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return fail(CCX_ECANCELLED, "server is shutting down");
        for (auto& kv : srv->jobs)
            if (kv.second->pr == pr && !kv.second->done)
                return fail(CCX_EINVAL, "problem already has a job in flight (ticket %llu)",
                            (unsigned long long)kv.first);
        j->ticket = srv->next_ticket++;
        j->run.gammas = j->gammas.data();
        srv->jobs[j->ticket] = j;
        srv->pending.push_back(j);
        *ticket = j->ticket;
    }
    srv->cv_work.notify_one();
    return CCX_OK;
}

ccx_status ccx_wait(ccx_server* srv, uint64_t ticket, int64_t timeout_ms) {
    g_err.clear();
    if (!srv) return fail(CCX_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) return fail(CCX_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    std::shared_ptr<ccx_server::Job> j = it->second;
    auto ready = [&] { return j->done; };
    if (timeout_ms < 0) srv->cv_done.wait(lk, ready);
    else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return fail(CCX_ETIMEOUT, "job %llu still running", (unsigned long long)ticket);
    srv->jobs.erase(ticket);
    if (j->status != CCX_OK) g_err = j->msg;
    return j->status;
}

ccx_status ccx_server_destroy(ccx_server* srv) {
    g_err.clear();
    if (!srv) return CCX_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        for (auto& j : srv->pending) {
            j->status = CCX_ECANCELLED;
            j->msg = "server destroyed before the job started";
            j->done = true;
        }
        srv->pending.clear();
    }
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    delete srv;
    return CCX_OK;
}


}  // extern "C"

// ------------------------------------------------------------------ feature shards
namespace {

// A problem used as one column shard of a larger problem: the gammas begun so
// far (for the predictor between gammas), the runner that begins them, and the
// norms of the whole problem that fix rho, eps and the error scale.
struct ShardState {
    PathRun run;
    std::vector<double> hist;
    double nyc = 0.0, ny0 = 0.0;
    bool open = false;
};

void drop_shard(ccx_problem* pr) {
    delete pr->shard;
    pr->shard = nullptr;
}

// make the caller's stream wait for the work stream without blocking the host
ccx_status leave_async(ccx_problem* pr) {
    CUDA_TRY(cudaEventRecord(pr->ev_done, pr->work));
    CUDA_TRY(cudaStreamWaitEvent(pr->user, pr->ev_done, 0));
    return CCX_OK;
}

template <typename R>
ccx_status shard_begin(ccx_problem* pr, ShardState& sh, double gamma) {
    PathRun& r = sh.run;
    if (!sh.open || !pr->path_started) {
        if (!pr->path_started) {
            const R* Y0 = std::is_same<R, double>::value ? reinterpret_cast<const R*>(pr->Y0d)
                                                          : reinterpret_cast<const R*>(pr->Y0f);
            CUDA_TRY(launch_pd_init<R>(make_params<R>(pr), Y0, pr->work));
            pr->path_started = true;
        }
        sh.hist.clear();
        r.conv_hist[0] = r.conv_hist[1] = r.conv_hist[2] = 0;
        r.all_conv = true;
        sh.open = true;
    }
    sh.hist.push_back(gamma);
    r.pr = pr;
    r.gammas = sh.hist.data();
    r.n_gamma = (int)sh.hist.size();
    r.g = r.n_gamma - 1;
    // rho, eps and the error floor come from the norms of the whole problem
    const double keep_c = pr->nyc, keep_0 = pr->ny0;
    pr->nyc = sh.nyc;
    pr->ny0 = sh.ny0;
    const ccx_status s = path_begin_gamma<R>(r);
    pr->nyc = keep_c;
    pr->ny0 = keep_0;
    return s;
}

template <typename R>
ccx_status shard_end(ccx_problem* pr, ShardState& sh, float* U_out, int32_t* labels_out, ccx_gamma_stats* stats) {
    PathRun& r = sh.run;
    IterParams<R> P = make_params<R>(pr);
    const bool u_dev = is_device_ptr(U_out), l_dev = is_device_ptr(labels_out);
    if (U_out) {
        if (u_dev) {
            CUDA_TRY(launch_pd_finalize<R>(P, U_out, pr->p, (int)pr->p, pr->work));
        } else {
            CUDA_TRY(launch_pd_finalize<R>(P, pr->Ustage, pr->p, (int)pr->p, pr->work));
            CUDA_TRY(cudaMemcpyAsync(U_out, pr->Ustage, sizeof(float) * pr->n * pr->p, cudaMemcpyDeviceToHost,
                                     pr->work));
        }
    }
    int* ldst = (labels_out && l_dev) ? labels_out : pr->Lstage;
    CUDA_TRY(launch_fused_labels((int)pr->n, P.m, pr->d_ei, pr->d_ej, pr->fused, ldst, pr->d_ncl, pr->cc_scratch,
                                 pr->work));
    if (labels_out && !l_dev)
        CUDA_TRY(cudaMemcpyAsync(labels_out, pr->Lstage, sizeof(int) * pr->n, cudaMemcpyDeviceToHost, pr->work));
    CUDA_TRY(cudaMemcpyAsync(pr->h_ncl, pr->d_ncl, sizeof(int), cudaMemcpyDeviceToHost, pr->work));
    CUDA_TRY(cudaMemcpyAsync(&pr->st_host[0], pr->st, sizeof(PdState), cudaMemcpyDeviceToHost, pr->work));
    CUDA_TRY(cudaStreamSynchronize(pr->work));
    const PdState f = pr->st_host[0];
    if (*pr->h_ncl < 0)
        return fail(CCX_ECUDA, "the connected-components pass over the fused edges did not settle within n + 1 "
                               "rounds; labels not written");
    r.conv_hist[2] = r.conv_hist[1];
    r.conv_hist[1] = r.conv_hist[0];
    r.conv_hist[0] = f.converged;
    if (stats) {
        stats->iters = f.iter;
        stats->converged = f.converged;
        stats->n_fused = std::max(f.n_fused, 0);
        stats->n_clusters = *pr->h_ncl;
        stats->gamma = r.gammas[r.g];
        stats->rho = r.rho;
        stats->eps = r.eps;
        stats->d_final = f.d_last;
        stats->err_est = f.err_est;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - r.t0).count();
        stats->n_recomputed = f.n_recomputed;
        stats->recomputes = f.recompute_total;
    }
    return CCX_OK;
}

}  // namespace

extern "C" {

ccx_status ccx_shard_norms(const ccx_problem* pr, double* yc_sq, double* y0_sq) {
    g_err.clear();
    if (!pr || !yc_sq || !y0_sq) return fail(CCX_EINVAL, "NULL argument");
    *yc_sq = pr->nyc * pr->nyc;
    *y0_sq = pr->ny0 * pr->ny0;
    return CCX_OK;
}

ccx_status ccx_shard_begin_gamma(ccx_problem* pr, double gamma, const ccx_opts* opts, double yc_sq_total,
                                 double y0_sq_total) {
    g_err.clear();
    if (!pr) return fail(CCX_EINVAL, "problem is NULL");
    if (!std::isfinite(gamma) || gamma < 0.0) return fail(CCX_EINVAL, "gamma must be finite and >= 0");
    if (!(yc_sq_total >= 0.0) || !(y0_sq_total >= 0.0) || !std::isfinite(yc_sq_total) || !std::isfinite(y0_sq_total))
        return fail(CCX_EINVAL, "the squared norms must be finite and >= 0");
    if (!pr->shard) pr->shard = new ShardState();
    ShardState& sh = *pr->shard;
    ccx_status s = resolve_opts(pr, opts, &sh.run.o);
    if (s != CCX_OK) return s;
    sh.run.o.anderson = 0;   // the shard calls run the plain iteration kernels only
    apply_opts(pr, sh.run.o);
    s = check_limits(pr);
    if (s != CCX_OK) return s;
    s = enter(pr);
    if (s != CCX_OK) return s;
    s = ensure_path(pr);
    if (s != CCX_OK) return s;
    sh.nyc = std::sqrt(yc_sq_total);
    sh.ny0 = std::sqrt(y0_sq_total);
    s = pr->precision == CCX_FP64 ? shard_begin<double>(pr, sh, gamma) : shard_begin<float>(pr, sh, gamma);
    if (s != CCX_OK) return s;
    return leave_async(pr);
}

ccx_status ccx_shard_partials(ccx_problem* pr, double* part, int64_t* len) {
    g_err.clear();
    if (!pr || !len) return fail(CCX_EINVAL, "NULL argument");
    const int64_t L = (int64_t)pr->le * kSliceThreads + kNumScalarPartials;
    if (!part) {
        *len = L;
        return CCX_OK;
    }
    if (!pr->shard || !pr->shard->open || !pr->path_ready)
        return fail(CCX_EINVAL, "ccx_shard_begin_gamma has not been called on this problem");
    if (*len < L) return fail(CCX_EINVAL, "part holds %lld doubles, %lld needed", (long long)*len, (long long)L);
    if (!is_device_ptr(part)) return fail(CCX_EINVAL, "part must be device memory");
    ccx_status s = enter(pr);
    if (s != CCX_OK) return s;
    if (pr->precision == CCX_FP64) {
        const IterParams<double> P = make_params<double>(pr);
        CUDA_TRY(launch_pd_slice_variant<double>(P, pr->variant, pr->work));
        CUDA_TRY(launch_pd_shard_partials<double>(P, part, pr->work));
    } else {
        const IterParams<float> P = make_params<float>(pr);
        CUDA_TRY(launch_pd_slice_variant<float>(P, pr->variant, pr->work));
        CUDA_TRY(launch_pd_shard_partials<float>(P, part, pr->work));
    }
    *len = L;
    return leave_async(pr);
}

ccx_status ccx_shard_reduce(ccx_problem* pr, const double* parts, int n_shards, int* done) {
    g_err.clear();
    if (!pr || !parts) return fail(CCX_EINVAL, "NULL argument");
    if (n_shards < 1) return fail(CCX_EINVAL, "n_shards must be >= 1");
    if (!pr->shard || !pr->shard->open || !pr->path_ready)
        return fail(CCX_EINVAL, "ccx_shard_begin_gamma has not been called on this problem");
    if (!is_device_ptr(parts)) return fail(CCX_EINVAL, "parts must be device memory");
    ccx_status s = enter(pr);
    if (s != CCX_OK) return s;
    const long long L = (long long)pr->le * kSliceThreads + kNumScalarPartials;
    if (pr->precision == CCX_FP64) {
        IterParams<double> P = make_params<double>(pr);
        P.ext_part = parts;
        P.n_ext = n_shards;
        P.ext_len = L;
        CUDA_TRY(launch_pd_reduce<double>(P, pr->work));
    } else {
        IterParams<float> P = make_params<float>(pr);
        P.ext_part = parts;
        P.n_ext = n_shards;
        P.ext_len = L;
        CUDA_TRY(launch_pd_reduce<float>(P, pr->work));
    }
    if (done) {
        CUDA_TRY(cudaMemcpyAsync(&pr->st_host[1], pr->st, sizeof(PdState), cudaMemcpyDeviceToHost, pr->work));
        CUDA_TRY(cudaStreamSynchronize(pr->work));
        *done = pr->st_host[1].done;
    }
    return leave_async(pr);
}

ccx_status ccx_shard_end_gamma(ccx_problem* pr, float* U_out, int32_t* labels_out, ccx_gamma_stats* stats) {
    g_err.clear();
    if (!pr) return fail(CCX_EINVAL, "problem is NULL");
    if (!pr->shard || !pr->shard->open || !pr->path_ready)
        return fail(CCX_EINVAL, "ccx_shard_begin_gamma has not been called on this problem");
    ccx_status s = enter(pr);
    if (s != CCX_OK) return s;
    s = pr->precision == CCX_FP64 ? shard_end<double>(pr, *pr->shard, U_out, labels_out, stats)
                                  : shard_end<float>(pr, *pr->shard, U_out, labels_out, stats);
    if (s != CCX_OK) return s;
    return leave(pr);
}

}  // extern "C"

namespace {
// n_iter MM iterations of the current warm-start state at penalty gamma with
// the stopping test off, each kernel launched alone between CUDA events on the
// work stream; mean milliseconds of the slice and reduce kernels.
// mix_ms: NULL (the plain map), or the mean time of the two Anderson mixing kernels, which then run
// after every iteration with history o.anderson (from the state the path holds, at this gamma)
ccx_status time_iterations_impl(ccx_problem* pr, double gamma, int n_iter, const ccx_opts& o, double* slice_ms,
                                double* reduce_ms, double* mix_ms = nullptr) {
    ccx_status s = check_limits(pr);
    if (s != CCX_OK) return s;
    s = enter(pr);
    if (s != CCX_OK) return s;
    s = ensure_path(pr);
    if (s != CCX_OK) return s;
    const int aa_m = mix_ms ? o.anderson : 0;
    if (aa_m > 0) {
        s = ensure_aa(pr);
        if (s != CCX_OK) return s;
    }
    const bool fp64 = pr->precision == CCX_FP64;
    double rho = o.rho_scale * (pr->nyc + gamma * pr->nw);
    if (!(rho > 0.0)) rho = o.rho_scale;
    double eps = (o.eps_rel * pr->nyc) * (o.eps_rel * pr->nyc);
    if (!(eps > 0.0)) eps = o.eps_rel * o.eps_rel;
    std::vector<cudaEvent_t> ev(4 * (size_t)n_iter);
    for (auto& e : ev) CUDA_TRY(cudaEventCreate(&e));
    auto body = [&](auto tag) -> ccx_status {
        using R = decltype(tag);
        IterParams<R> P = make_params<R>(pr);
        if (!pr->path_started) {
            const R* Y0 = fp64 ? reinterpret_cast<const R*>(pr->Y0d) : reinterpret_cast<const R*>(pr->Y0f);
            CUDA_TRY(launch_pd_init<R>(P, Y0, pr->work));
            pr->path_started = true;
        }
        // tol < 0: neither stopping rule fires; max_iter leaves room for all iterations
        CUDA_TRY(launch_pd_begin_gamma<R>(P, gamma, rho, eps, -1.0, n_iter + 1, o.accelerate, 0.0, aa_m,
                                          pr->work));
        for (int k = 0; k < n_iter; ++k) {
            CUDA_TRY(cudaEventRecord(ev[4 * k], pr->work));
            CUDA_TRY(launch_pd_slice_variant<R>(P, pr->variant, pr->work));
            CUDA_TRY(cudaEventRecord(ev[4 * k + 1], pr->work));
            CUDA_TRY(launch_pd_reduce<R>(P, pr->work));
            CUDA_TRY(cudaEventRecord(ev[4 * k + 2], pr->work));
            if (aa_m > 0) CUDA_TRY(launch_pd_aa<R>(P, pr->work));
            CUDA_TRY(cudaEventRecord(ev[4 * k + 3], pr->work));
        }
        CUDA_TRY(cudaStreamSynchronize(pr->work));
        double a = 0.0, b = 0.0, c = 0.0;
        for (int k = 0; k < n_iter; ++k) {
            float t1 = 0.f, t2 = 0.f, t3 = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&t1, ev[4 * k], ev[4 * k + 1]));
            CUDA_TRY(cudaEventElapsedTime(&t2, ev[4 * k + 1], ev[4 * k + 2]));
            CUDA_TRY(cudaEventElapsedTime(&t3, ev[4 * k + 2], ev[4 * k + 3]));
            a += t1;
            b += t2;
            c += t3;
        }
        *slice_ms = a / n_iter;
        *reduce_ms = b / n_iter;
        if (mix_ms) *mix_ms = c / n_iter;
        return CCX_OK;
    };
    s = fp64 ? body(double{}) : body(float{});
    for (auto& e : ev) cudaEventDestroy(e);
    if (s != CCX_OK) return s;
    return leave(pr);
}
}  // namespace

extern "C" {

ccx_status ccx_time_iterations(ccx_problem* pr, double gamma, int n_iter, const ccx_opts* opts, double* slice_ms,
                               double* reduce_ms) {
    g_err.clear();
    if (!pr || !slice_ms || !reduce_ms) return fail(CCX_EINVAL, "NULL argument");
    if (!std::isfinite(gamma) || gamma < 0.0) return fail(CCX_EINVAL, "gamma must be finite and >= 0");
    if (n_iter < 1) return fail(CCX_EINVAL, "n_iter must be >= 1");
    ccx_opts o;
    ccx_status s = resolve_opts(pr, opts, &o);
    if (s != CCX_OK) return s;
    apply_opts(pr, o);
    return time_iterations_impl(pr, gamma, n_iter, o, slice_ms, reduce_ms);
}

ccx_status ccx_time_iterations_mixing(ccx_problem* pr, double gamma, int n_iter, const ccx_opts* opts,
                                      double* slice_ms, double* reduce_ms, double* mix_ms) {
    g_err.clear();
    if (!pr || !opts || !slice_ms || !reduce_ms || !mix_ms) return fail(CCX_EINVAL, "NULL argument");
    if (!std::isfinite(gamma) || gamma < 0.0) return fail(CCX_EINVAL, "gamma must be finite and >= 0");
    if (n_iter < 1) return fail(CCX_EINVAL, "n_iter must be >= 1");
    ccx_opts o;
    ccx_status s = resolve_opts(pr, opts, &o);
    if (s != CCX_OK) return s;
    if (o.anderson < 1) return fail(CCX_EINVAL, "opts->anderson must be >= 1 to time the mixing kernels");
    apply_opts(pr, o);
    return time_iterations_impl(pr, gamma, n_iter, o, slice_ms, reduce_ms, mix_ms);
}

ccx_status ccx_tune_grid(ccx_problem* pr, int g_min, int* g_out, double* ms_out) {
    g_err.clear();
    if (!pr || !g_out) return fail(CCX_EINVAL, "NULL argument");
    if (pr->path_started)
        return fail(CCX_EINVAL, "ccx_tune_grid runs iterations from Y_0: call it before the first solve or after "
                                "ccx_reset_path");
    if (pr->ei.empty()) return fail(CCX_EINVAL, "no edges");
    ccx_opts o;
    ccx_status s = resolve_opts(pr, nullptr, &o);
    if (s != CCX_OK) return s;
    pr->tuned_G = 0;
    const int gmax = grid_of_cap(pr, 0);
    const int lo = std::max(1, std::min(g_min, gmax));
    int best = gmax;
    double best_cost = 0.0, best_ms = 0.0;
    for (int G = gmax; G >= lo; G = (G == lo) ? 0 : std::max(lo, G / 2)) {
        o.max_ctas = G;
        apply_opts(pr, o);
        double a = 0.0, b = 0.0;
        pr->path_started = false;
        s = time_iterations_impl(pr, 0.0, 3, o, &a, &b);      // warm-up: kernel attributes, caches
        if (s == CCX_OK) s = time_iterations_impl(pr, 0.0, 16, o, &a, &b);
        if (s != CCX_OK) {
            pr->path_started = false;
            return s;
        }
        const double ms = a + b;
        const double cost = ms * G;                            // SM-milliseconds per iteration
        // a smaller grid must save a good part of the SM time: when the cost is only
        // level (a work-bound problem), a small grid leaves a batch a long tail in
        // which the last problems run on few SMs
        if (G == gmax || cost < best_cost * 0.7) {
            best = G;
            best_cost = cost;
            best_ms = ms;
        }
    }
    pr->path_started = false;                                  // the next solve starts from Y_0
    pr->tuned_G = best == gmax ? 0 : best;
    *g_out = best;
    if (ms_out) *ms_out = best_ms;
    return CCX_OK;
}

uint64_t ccx_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

ccx_status ccx_reset_path(ccx_problem* pr) {
    g_err.clear();
    if (!pr) return fail(CCX_EINVAL, "problem is NULL");
    pr->path_started = false;
    pr->last_fused = -1;
    if (pr->shard) pr->shard->open = false;
    return CCX_OK;
}

ccx_status ccx_problem_destroy(ccx_problem* pr) {
    g_err.clear();
    if (!pr) return CCX_OK;
    cudaSetDevice(pr->device);
    cudaStreamSynchronize(pr->work);
    free_all(pr);
    drop_shard(pr);
    delete pr;
    return CCX_OK;
}

}  // extern "C"
