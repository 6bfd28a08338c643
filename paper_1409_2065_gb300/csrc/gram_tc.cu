// Gram matrix G = Y Y^T of the kNN weight rule (Calibration of Weights, Eq. 8:
// d2_ij = ||y_i||^2 + ||y_j||^2 - 2 <y_i, y_j>) on the 5th-generation tensor
// cores, accumulating in FP32 in tensor memory: tcgen05.mma kind::tf32 reading
// FP32 rows straight from shared memory, or kind::f16 on BF16 rows (a copy of Y
// rounded to nearest BF16 by a conversion kernel).  In both cases a stage holds
// 128 bytes of every row, i.e. 32 TF32 or 64 BF16 values, and takes four MMAs
// of K = 8 (TF32) or K = 16 (BF16).
//
// One CTA per 128 x 128 output tile of the upper triangle (the lower one is
// written as its mirror).  Warp 0 lane 0 streams 128-row tiles of Y, 128 bytes
// per row (128-byte swizzle), into a 4-stage ring with TMA; warp 1 lane 0
// issues the stage's four 128 x 128 MMAs and returns each stage to the
// producer with tcgen05.commit; all four warps then read the accumulator out of
// tensor memory (tcgen05.ld, one 32-lane quarter per warp).  Every wait is
// bounded: on a timeout the kernel raises an error flag, releases its tensor
// memory and returns, and the host reports the failure.
//
// The products are formed from TF32- or BF16-rounded inputs, so the result is
// an approximation with a stated error bound (returned through `unit`); the
// kNN rule uses it only to select candidates and recomputes their distances
// exactly, so the edge set does not depend on which input rounding was used.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>

#include "ccx_internal.h"

namespace ccx {
namespace {

constexpr int kBM = 128, kBN = 128;       // output tile
constexpr int kRowBytes = 128;            // bytes of a row per stage: one swizzle row
constexpr int kMmaBytes = 32;             // K bytes of one MMA (8 TF32 or 16 BF16 values)
constexpr int kStages = 4;
constexpr int kTileBytes = kBM * kRowBytes; // 16 KB per operand tile
constexpr int kStageBytes = 2 * kTileBytes;
constexpr int kThreads = 128;
constexpr uint32_t kTmemCols = 128;       // 128 lanes x 128 FP32 columns
constexpr uint32_t kSpinLimit = 1u << 24; // polls of an mbarrier before giving up
constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes + 1024 /*alignment*/ + 256 /*barriers*/;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait on the phase with the given parity; false (and the error flag) on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* fail) {
    for (uint32_t k = 0; k < kSpinLimit; ++k) {
        if (mbar_test(bar, parity)) return true;
        if (*fail) return false;
    }
    *fail = 1;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA with
// the 128-byte swizzle: rows 128 bytes apart, 8-row groups 1024 bytes apart
// (stride byte offset), leading byte offset unused for this layout, version 1,
// layout type 2 (128-byte swizzle).  The tile base is 1024-byte aligned, so a
// K step inside the swizzle row is a plain byte offset of the start address.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;           // leading byte offset (16 B units; ignored here)
    d |= (uint64_t)(1024u >> 4) << 32; // stride byte offset
    d |= (uint64_t)1u << 46;           // descriptor version
    d |= (uint64_t)2u << 61;           // 128-byte swizzle
    return d;
}

// Instruction descriptors: FP32 accumulator, A and B both K-major, N = 128,
// M = 128; operand format 2 = TF32 (kind::tf32), 1 = BF16 (kind::f16).
constexpr uint32_t instr_desc(uint32_t ab_format) {
    return (1u << 4)                        // D format: F32
           | (ab_format << 7)               // A format
           | (ab_format << 10)              // B format
           | ((uint32_t)(kBN >> 3) << 17)   // N / 8
           | ((uint32_t)(kBM >> 4) << 24);  // M / 16
}

template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, int n, int ktiles, float* __restrict__ G,
                   int* __restrict__ err) {
    constexpr int kBK = BF16 ? 64 : 32;    // values per row per stage (128 bytes)
    constexpr uint32_t kInstrDesc = instr_desc(BF16 ? 1u : 2u);
    const int bm = blockIdx.y, bn = blockIdx.x;
    if (bn < bm) return;   // the lower triangle is written as the mirror of the upper one
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* fail = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int kt = 0; kt < ktiles; ++kt) {
            const int s = kt % kStages;
            const uint32_t use = (uint32_t)(kt / kStages);
            if (kt >= kStages && !mbar_wait(&empty[s], (use & 1u) ^ 1u, fail)) break;
            unsigned char* a = sm + (size_t)s * kStageBytes;
            mbar_expect_tx(&full[s], kStageBytes);
            tma_load_2d(a, &tmap, kt * kBK, bm * kBM, &full[s]);
            tma_load_2d(a + kTileBytes, &tmap, kt * kBK, bn * kBN, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int kt = 0; kt < ktiles; ++kt) {
            const int s = kt % kStages;
            if (!mbar_wait(&full[s], (uint32_t)(kt / kStages) & 1u, fail)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a = smem_u32(sm + (size_t)s * kStageBytes);
            const uint32_t b = a + kTileBytes;
#pragma unroll
            for (int kk = 0; kk < kRowBytes / kMmaBytes; ++kk) {
                const uint64_t da = smem_desc_sw128(a + kk * kMmaBytes);
                const uint64_t db = smem_desc_sw128(b + kk * kMmaBytes);
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                if constexpr (BF16) {
                    asm volatile(
                        "{\n"
                        ".reg .pred p;\n"
                        "setp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
                        "}\n" ::"r"(tmem),
                        "l"(da), "l"(db), "r"(kInstrDesc), "r"(acc)
                        : "memory");
                } else {
                    asm volatile(
                        "{\n"
                        ".reg .pred p;\n"
                        "setp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
                        "}\n" ::"r"(tmem),
                        "l"(da), "l"(db), "r"(kInstrDesc), "r"(acc)
                        : "memory");
                }
            }
            // the stage goes back to the producer once these MMAs have read it
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(done))
                     : "memory");
    }
    __syncwarp();

    // epilogue: warp w owns accumulator lanes (tile rows) 32 w .. 32 w + 31
    const bool ok = mbar_wait(done, 0u, fail);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && !*fail) {
        const int row = bm * kBM + warp * 32 + lane;
        for (int c0 = 0; c0 < kBN; c0 += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                "[%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int col = bn * kBN + c0 + j;
                const float v = __uint_as_float(r[j]);
                if (row < n && col < n) {
                    G[(size_t)row * n + col] = v;
                    if (bm != bn) G[(size_t)col * n + row] = v;
                }
            }
        }
    }
    if (*fail && lane == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// rows of Y rounded to nearest BF16 (n x ld; the padding columns stay 0)
__global__ void to_bf16_kernel(const float* __restrict__ Y, size_t total, __nv_bfloat16* __restrict__ Yb) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x)
        Yb[k] = __float2bfloat16_rn(Y[k]);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            (void)cudaGetLastError();
    });
    return fn;
}

}  // namespace

cudaError_t launch_gram_tc(const float* Y, int n, int p, int ld, float* G, double* unit, cudaStream_t s, int bf16) {
    int dev = 0, major = 0, minor = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (e != cudaSuccess) return e;
    if (major != 10 || n < 1 || ld % 32 != 0 || (reinterpret_cast<uintptr_t>(Y) & 15u) != 0)
        return cudaErrorNotSupported;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int kbk = bf16 ? 64 : 32;                      // values per 128-byte stage row
    const size_t esz = bf16 ? 2 : 4;
    __nv_bfloat16* Yb = nullptr;
    const void* base = Y;
    if (bf16) {
        if ((e = cudaMallocAsync(&Yb, sizeof(__nv_bfloat16) * (size_t)n * ld, s)) != cudaSuccess) return e;
        const size_t total = (size_t)n * ld;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 8192) blocks = 8192;
        count_launches(1);
        to_bf16_kernel<<<blocks, 256, 0, s>>>(Y, total, Yb);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            cudaFreeAsync(Yb, s);
            return e;
        }
        base = Yb;
    }
    // Y as a 2-D tensor: inner dimension ld columns (the padding columns are 0),
    // outer n rows; boxes of 128 bytes x 128 rows, entries past n (or past ld in
    // the last BF16 stage) read as 0
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * esz};
    const cuuint32_t box[2] = {(cuuint32_t)kbk, (cuuint32_t)kBM};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
            const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        if (Yb) cudaFreeAsync(Yb, s);
        return cudaErrorNotSupported;
    }
    auto kern = bf16 ? gram_tc_kernel<true> : gram_tc_kernel<false>;
    static int attr_set[2] = {0, 0};
    if (!attr_set[bf16 ? 1 : 0]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        if (e != cudaSuccess) {
            if (Yb) cudaFreeAsync(Yb, s);
            return e;
        }
        attr_set[bf16 ? 1 : 0] = 1;
    }
    int* err = nullptr;
    if ((e = cudaMallocAsync(&err, sizeof(int), s)) != cudaSuccess) {
        if (Yb) cudaFreeAsync(Yb, s);
        return e;
    }
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), s)) != cudaSuccess) return e;
    const int nt = (n + kBM - 1) / kBM;
    const int ktiles = (ld + kbk - 1) / kbk;
    count_launches(1);
    kern<<<dim3(nt, nt), kThreads, kSmemBytes, s>>>(map, n, ktiles, G, err);
    e = cudaGetLastError();
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(err, s);
    if (Yb) cudaFreeAsync(Yb, s);
    if (e != cudaSuccess) return e;
    if (herr) return cudaErrorLaunchTimeout;   // a bounded wait gave up: no result
    // |G_ij - <y_i, y_j>| <= unit ||y_i|| ||y_j||: the rounded operands (TF32:
    // the low mantissa bits dropped, relative error below 2^-10 each, so 2^-9 +
    // 2^-20 per product; BF16: rounded to nearest, below 2^-8 each, so 2^-7 +
    // 2^-16 per product), Cauchy-Schwarz over the row, the float rounding of
    // the filled rows (2 * 2^-24) and FP32 accumulation over ld terms, allowed
    // 4 units of 2^-24 per addition
    const double prod = bf16 ? 1.0 / 128.0 + 1.0 / 65536.0 : 1.0 / 512.0 + 1.0 / 1048576.0;
    *unit = prod + 2.0 / 16777216.0 + (double)(ld + 64) * 4.0 / 16777216.0;
    (void)p;
    return cudaSuccess;
}

}  // namespace ccx
