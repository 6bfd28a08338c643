// Internal declarations of the ccx library (not part of the C ABI).
//
// Data layout on the device (one problem):
//   * every n x p matrix is row-major with an internal row stride ld that is
//     p rounded up to a multiple of 32 elements; padding columns hold 0 and
//     stay 0 through every kernel;
//   * the observation mask is bit-packed, n rows of ld/32 words, bit = 1 for
//     observed (padding columns are marked observed);
//   * the projection A of the MM iteration is kept in float-float (hi + lo
//     float arrays) for the FP32 path and in double for the FP64 path; all
//     other per-entry quantities are in the path's real type R.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ccx.h"

namespace ccx {

constexpr int kSliceThreads = 512;   // threads of the fused iteration kernel
constexpr int kSliceCols = 4;        // columns per staged slice (one 16-byte vector for float)
constexpr int kReduceThreads = 256;
constexpr int kConvWindow = 64;      // iterations per convergence window
constexpr int kRateWindows = 8;      // windows spanned by the contraction-rate estimate
constexpr int kNumScalarPartials = 8;
constexpr double kStallSteps = 128.0;  // error bound, in steps, once steps are at the rounding level
constexpr double kNoiseFactor = 8.0;   // steps within this factor of the rounding noise: no progress possible
constexpr int kNoiseWindows = 8;       // consecutive such windows before stopping
constexpr int kStallWindows = 16;      // windows without a 2x residual decrease over kRateWindows before a plateau exit
constexpr double kStallTolFactor = 100.0;  // a plateau exit needs the rate-based error estimate within this x tol
constexpr double kFuseMargin = 1e-5;   // relative margin of a "clearly fused" edge (mu w d >= rho ||b|| (1 + margin))
constexpr int kAaMax = 16;             // longest history of the Anderson mixing
constexpr int kAaBudget = 3000;        // mixing iterations of one gamma before the hand-over
constexpr int kAaDots = 2 * kAaMax + 3;  // partial sums per block of pd_aa_update_kernel

// Scalar partial slots written by each CTA of the iteration kernel.
enum : int {
    kPsUA = 0,     // ||U_y - A_m||^2
    kPsVB = 1,     // ||V_y - B_m||^2
    kPsRestart = 2,// <a_start - A_m, A_m - A_{m-1}> (restart test)
    kPsStep = 3,   // ||A_m - A_{m-1}||^2
    kPsNormA = 4,  // ||A_m||^2
    kPsNoise = 5,  // sum of ((|U_y - A_start| + |G|) / (1 + deg))^2: rounding scale of the step
    kPsDelta = 6,  // ||A_m - A_start||^2: residual of the map at the extrapolated point
};

// Device-resident scalar state of the MM iteration of one problem.  Written
// by the host only between gammas (through pd_begin_gamma) and otherwise by
// the last block of pd_reduce_kernel.
struct PdState {
    double alpha1;        // alpha_{m-1} = d_{m-1} / (d_{m-1} + rho_{m-1})
    double alpha2;        // alpha_{m-2}
    double beta;          // extrapolation weight used by the next iteration
    double gamma, rho, eps, tol;
    double d_last;
    double blk_max, err_est, a_norm;
    double scale_floor;   // lower bound of the error scale (rounding level of the data)
    double noise_max;     // window maximum of the rounding-noise scale of the step
    double dmax;          // window maximum of ||A_m - A_start|| (the map's residual)
    double ring[kRateWindows];  // recent window maxima of that residual
    double g_last;        // last measured residual decay rate per iteration (0: none yet)
    int ring_len;
    int floor_hits;       // consecutive windows with steps at the rounding level
    int stall_hits;       // consecutive windows in which the residual made no 2x progress
    unsigned long long fused_hash;   // order-free hash of the clearly fused edges
    int k_mom;
    int accelerate;
    int par;              // slot parity: input slots of the next iteration
    int iter;             // iterations done on the current gamma
    int max_iter;
    int done;             // current gamma finished
    int converged;        // 1: tolerance met, 2: stopped at the rounding floor
    int hits;             // consecutive windows that met the tolerance
    int n_fused;
    int fused_stable;     // iterations since the fused set last changed
    unsigned int counter; // arrival counter of the reduce kernel's blocks
    int n_recomputed;     // edges of the last iteration whose fuse decision came from the FP64 recompute
    long long recompute_total;  // FP64 recomputes over the current gamma's iterations
    // Anderson mixing of the MM map (aa_kernels.cu): the state z = (A, t, alpha) of
    // an iteration is replaced by a combination of the last aa_m map outputs, from
    // the start of a gamma until the hand-over to the restart rule
    int aa_m;             // history length (0: no mixing in this problem)
    int aa_on;            // mixing active in the current gamma
    int aa_len;           // history entries held (<= aa_m)
    int aa_head;          // ring slot the next entry takes
    int aa_iters;         // iterations of the current mixing phase
    int aa_have_prev;     // the previous iteration's residual is held
    unsigned int aa_counter;  // arrival counter of pd_aa_update_kernel's blocks
    int aa_total;         // mixing iterations of the current gamma (reported)
    double aa_M[kAaMax][kAaMax];  // Gram matrix of the residual differences, by ring slot
    double aa_g[kAaMax];          // mixing coefficients of the next mix, by ring slot (0 off the history)
    double aa_win[4];             // residual norm at the ends of the last four windows
    double aa_ra_prev;            // alpha part of the previous residual
    double aa_sa;                 // alpha part of the last step z_k - z_(k-1)
    double aa_RA[kAaMax], aa_GA[kAaMax];  // alpha parts of the ring entries
};

template <typename R>
struct IterParams {
    const R* X;                 // n x ld data (observed entries; 0 elsewhere)
    const uint32_t* mask;       // n x ldw bits, or nullptr (all observed)
    R* Ahi[2];                  // A slots (hi part, or the double value)
    float* Alo[2];              // A slots (lo part; FP32 path only)
    R* Dl[2];                   // velocity slots Delta = A_m - A_{m-1}
    R* Q;                       // missing entries: U_y - A of the last iteration
    R* Em;                      // missing entries: U - A_prev of the last iteration
    // The two edge sweeps of the iteration kernel are split into equal runs,
    // one per thread: thread t takes node-sweep entries (CSR positions over
    // both directions) [t*la, (t+1)*la) and edge-sweep entries (edge ids in
    // (i, j) order) [t*le, (t+1)*le), the entries of each row of a run in an
    // order chosen against shared-memory bank conflicts.  Per-entry arrays of
    // a sweep store the k-th entry of thread t at k*T + t (T = kSliceThreads),
    // so a warp's k-th step reads consecutive words.
    R* t[2];                    // (t_m, t_{m-1}) pairs, t = 1 - s: la*T pairs in node-sweep
                                // order, then le*T pairs in edge-sweep order
    const int* rowptr;          // CSR over both directions, n + 1
    const int* erow;            // n + 1: first edge whose smaller endpoint is i
    const int* ps0;             // n + 1: first node-sweep partial slot of node i
    const uint16_t* csrT;       // la*T: neighbour of each node-sweep entry
    const uint16_t* ejT;        // le*T: larger endpoint of each edge-sweep entry
    const uint2* thrA;          // T: (node of the first entry, first partial slot) of each node-sweep run
    const int* thrE;            // T: smaller endpoint of the first edge of each edge-sweep run
    const int2* posA;           // le*T: node-sweep positions of the edge at each edge-sweep position
    const int* eid;             // le*T: edge id at each edge-sweep position (-1: padding)
    const int* ei;              // edge endpoints, i < j
    const int* ej;
    const double* w;            // edge weights
    float* Pnb;                 // per-CTA per-edge partial ||b||^2, G x le*T (edge-sweep order)
    double* Ps;                 // per-CTA scalar partials, G x kNumScalarPartials
    double* nb;                 // per-edge ||b_m|| of the last iteration
    uint8_t* fused;             // per-edge fused flag of t_{m+1}
    unsigned long long* Rf;     // per reduce-block fused count / hash
    PdState* st;
    // Near-threshold recompute (V update of the paper: the prox returns zero when
    // mu w d >= rho ||b||): an edge whose two sides differ by at most
    // delta_fuse * rho ||b|| has ||b_ij|| recomputed in double from the rows of
    // A_m before the decision; 0 disables it.
    double delta_fuse;
    // Feature-sharded iteration: when ext_part is set, the reduction takes each
    // edge-sweep position's ||b||^2 and the scalar partials from n_ext shards'
    // partial vectors (shard s at ext_part + s * ext_len: le*T per-position
    // doubles, then kNumScalarPartials doubles), summed in shard order, instead
    // of this problem's per-CTA partials.
    const double* ext_part;
    int n_ext;
    long long ext_len;
    // Anderson mixing buffers (float): aa_m rings of residual differences and of
    // map-output differences for A (n*ld each) and t (le*T each, edge-sweep order),
    // the last step z_k - z_(k-1) (A and t parts), the previous residual's t part,
    // and the per-block partial sums of pd_aa_update_kernel
    float* aaR;
    float* aaG;
    float* aaS;
    float* aaRt;
    float* aaGt;
    float* aaSt;
    float* aaPt;
    double* aaP;
    int aa_blocks;
    int aa_hist;                // history length of the mixing buffers (selects the kernels' ring bound)
    int n, p, ld, ldw, m, nslices, G;
    int la, le, nslots;         // run lengths of the two sweeps; node-sweep partial slots
    int stream_edges;           // 1: per-entry arrays of the sweeps stay in global memory
};

// ---------------------------------------------------------------- launchers
// (defined in pd_kernels.cu; all asynchronous on `s`)
template <typename R>
cudaError_t launch_pd_init(const IterParams<R>& P, const R* Y0, cudaStream_t s);
// aa_m > 0 starts the gamma with an Anderson mixing phase of history aa_m
template <typename R>
cudaError_t launch_pd_begin_gamma(const IterParams<R>& P, double gamma, double rho, double eps, double tol,
                                  int max_iter, int accelerate, double scale_floor, int aa_m, cudaStream_t s);
template <typename R>
cudaError_t launch_pd_iteration(const IterParams<R>& P, cudaStream_t s);
template <typename R>
cudaError_t launch_pd_slice(const IterParams<R>& P, cudaStream_t s);
template <typename R>
cudaError_t launch_pd_reduce(const IterParams<R>& P, cudaStream_t s);
// library-wide count of kernel launches (incremented by every launcher)
void count_launches(unsigned long long k);
template <typename R>
cudaError_t launch_pd_extrapolate(const IterParams<R>& P, R* p1_hi, float* p1_lo, R* p2_hi, float* p2_lo, double w0,
                                  double w1, double w2, cudaStream_t s);
template <typename R>
cudaError_t launch_pd_finalize(const IterParams<R>& P, float* U_out, int64_t ld_out, int p, cudaStream_t s);
size_t pd_slice_smem_bytes(int n, int la, int le, int nslots, bool fp64, bool prefetch, bool stream);
// iteration-kernel variant: 0 automatic, 1 double-buffered staging where it fits, 2 single buffer
template <typename R>
cudaError_t launch_pd_slice_variant(const IterParams<R>& P, int variant, cudaStream_t s);
template <typename R>
cudaError_t launch_pd_iteration_variant(const IterParams<R>& P, int variant, cudaStream_t s);
// Anderson mixing (aa_kernels.cu), launched after the reduction of every iteration;
// both kernels return at once unless the current gamma is in its mixing phase
template <typename R>
cudaError_t launch_pd_aa(const IterParams<R>& P, cudaStream_t s);
// per-position and scalar partials of this problem's CTAs, summed over CTAs in a
// fixed order into out (le*T + kNumScalarPartials doubles): one shard's share
template <typename R>
cudaError_t launch_pd_shard_partials(const IterParams<R>& P, double* out, cudaStream_t s);
int pd_reduce_blocks(int le);

// data preparation (prep_kernels.cu)
cudaError_t launch_pack_input(const float* X, const uint8_t* mask, int64_t n, int64_t p, int64_t ld_in,
                              float* Xf, double* Xd, uint32_t* maskbits, int ld, int ldw, int* bad_count,
                              cudaStream_t s);
cudaError_t launch_standardize(float* Xf, double* Xd, const uint32_t* maskbits, int n, int p, int ld, int ldw,
                               double* work, cudaStream_t s);
cudaError_t launch_fill_missing(const float* Xf, const double* Xd, const uint32_t* maskbits, int n, int p,
                                int ld, int ldw, double* colmean, float* Y0f, double* Y0d, double* ss,
                                cudaStream_t s);

// connected components of the fused edges (cc_kernels.cu)
cudaError_t launch_fused_labels(int n, int m, const int* ei, const int* ej, const uint8_t* fused,
                                int* labels, int* n_clusters, int* scratch, cudaStream_t s);

// per-edge fusion ratios into the library's fixed device buffer (static_scratch.cu)
constexpr int kStaticEdgesMax = 1 << 20;   // 8 MiB of doubles per device
// device address of the buffer on the current device (looked up once per device)
cudaError_t static_edge_scratch(double** out);
cudaError_t edge_ratios_static(const float* Y0f, int p, int ld, const int* ei_d, const int* ej_d, const double* w_d,
                               int m, double* scratch, cudaStream_t s);

// kNN weights (knn_kernels.cu)
struct KnnResult {
    std::vector<int> ei, ej;
    std::vector<double> w, d2;
    double phi = 0.0;
};
// geo: NULL (Euclidean rule), or device (latitude, longitude) pairs in degrees for the
// composite distance alpha ||y_i - y_j|| + (1 - alpha) g_ij (geodesic: great-circle g)
// gram: 0 tensor cores on TF32 operands, 1 tensor cores on BF16 operands, 2 FP32 CUDA cores
cudaError_t knn_build(const float* Y0f, int n, int p, int ld, int k, double phi, int phi_auto, int normalize,
                      cudaStream_t s, KnnResult* out, std::string* err, const double* geo = nullptr,
                      double alpha = 1.0, int geodesic = 0, int gram = 0);
// union of the kNN lists (nbr, nd2: device, n x kk, from knn_build's list pass), phi and the
// weights on the device (knn_weights.cu); the edges come back to the host sorted by (ei, ej)
cudaError_t knn_union_weights(const int* nbr, const double* nd2, int n, int kk, double phi, int phi_auto,
                              int normalize, cudaStream_t s, KnnResult* out);
// principal axes of Y_0 (pc_kernels.cu): axes q x p doubles (device), variances on the host
int pc_max_axes();
cudaError_t pc_axes(const float* Y0f, const double* mean, int n, int p, int ld, int q, double* axes, double* var_h,
                    cudaStream_t s);
// S (n x q floats, device) = (U - mean) axes^T for U n x ldu floats (device)
cudaError_t pc_project(const float* U, int ldu, const double* mean, const double* axes, int n, int p, int q, float* S,
                       cudaStream_t s);

// smallest k in [1, k_max] whose kNN union graph is connected (0: none), by
// bisection over GPU connected components of the k-prefix of the neighbour lists
cudaError_t knn_min_connected_k(const float* Y0f, int n, int p, int ld, int k_max, cudaStream_t s, int* k_out,
                                int* probes, std::string* err);
cudaError_t edge_distances(const float* Y0f, int n, int p, int ld, const int* ei_d, const int* ej_d, int m,
                           double* d2_d, cudaStream_t s);

}  // namespace ccx
