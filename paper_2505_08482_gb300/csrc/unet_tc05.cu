// BF16 GEMM of the warm-start network on the fifth-generation tensor cores:
// C[M][N] = A[M][K] . B[N][K]^T (+ bias[n]) (ReLU), FP32 accumulation in tensor
// memory, the same contract as the warp-level GEMM of unet_kernels.cu.
//
// One CTA of four warps computes a 128 x 128 tile of C.  Operand tiles of 128 rows x 64
// K-elements (128 bytes per row) are copied by the tensor memory accelerator from global
// memory into shared memory with the 128-byte swizzle, in a ring of STAGES buffers
// guarded by "full" and "empty" mbarriers.  One thread issues the copies, one thread
// issues the 128 x 128 x 16 MMAs (tcgen05.mma, kind::f16, A and B both BF16) into a
// 128-column FP32 accumulator in tensor memory and commits each stage back to its
// "empty" barrier; after the last stage a commit on the "done" barrier releases the
// epilogue, in which warp w reads accumulator lanes 32w..32w+31 (one row of C per
// thread) with tcgen05.ld, adds the bias, applies the ReLU and stores bf16 / fp32 or
// adds fp32 atomically (split K).
//
// Every mbarrier wait is bounded (kWaitNs of %globaltimer time).  A wait that gives up
// sets the CTA's abort flag and bit PAT_STATUS_TC05 of the caller's status word;
// the CTA then waits (bounded) for the copies it issued, frees its tensor memory and
// returns without storing: no hang, and the caller sees the flag.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "pat_internal.h"
#include "sync.cuh"
#include "unet.h"

namespace pat {
namespace tc05 {

constexpr int BM = 128, BK = 64, STAGES = 4, THREADS = 128;
constexpr uint32_t TILE_A = BM * BK * 2;            // bytes of one A tile (128 rows x 64 K-elements)
constexpr uint64_t kWaitNs = 200000000ull;          // 0.2 s per wait
constexpr int GROUP_M = 8;                          // tile rows per group of the tile order

// Shared memory of a CTA with an N tile of BN: the 4-stage ring of A and B tiles (1024-byte
// aligned for the 128-byte swizzle) and the barriers.
template <int BN>
__host__ __device__ constexpr size_t smem_bytes() {
    return 1024 + size_t(STAGES) * (TILE_A + uint32_t(BN) * BK * 2) + 256;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at bits 17-22,
// M / 16 at bits 24-28.
template <int BN>
__host__ __device__ constexpr uint32_t idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(BM >> 4) << 24);
}

// Shared-memory matrix descriptor of a K-major tile with the 128-byte swizzle: start
// address / 16 (bits 0-13), leading byte offset / 16 (bits 16-29; not used by swizzled
// K-major tiles), stride byte offset / 16 = 1024 / 16 (bits 32-45: 8 rows of 128 bytes),
// descriptor version 1 (bits 46-47), swizzle mode 2 = 128 bytes (bits 61-63).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
           (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* mb) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            s_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(s_addr(mb))
        : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(id), "r"(acc)
        : "memory");
}

// arrive on mb once every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* mb) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_addr(mb))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

struct Args {
    int M, N, K;
    int ksplit;            // K range per blockIdx.z (a multiple of BK)
    const float* bias;     // [N] or null
    int relu;
    void* C;
    int ldc;
    int out_mode;          // 0 bf16 store, 1 fp32 store, 2 fp32 atomic add
    int* status;           // device status word (bit PAT_STATUS_TC05 on a given-up wait), or null
};

// grid.x: output tiles in groups of GROUP_M tile rows (within a group the tile row varies
// fastest, so that CTAs running at the same time share A and B tiles in L2); grid.z: K split.
template <int BN>
__global__ void __launch_bounds__(THREADS, 1) k_gemm_tc05(const __grid_constant__ CUtensorMap ta,
                                                          const __grid_constant__ CUtensorMap tb, Args a) {
    constexpr uint32_t TILE_B = uint32_t(BN) * BK * 2;
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    unsigned char* sA = sm;
    unsigned char* sB = sm + STAGES * TILE_A;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * TILE_B);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    int* issued = const_cast<int*>(abort_flag) + 1;   // copies issued by the producer
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = (a.M + BM - 1) / BM, tiles_n = (a.N + BN - 1) / BN;
    const int t = blockIdx.x;
    const int first_m = (t / (GROUP_M * tiles_n)) * GROUP_M;
    const int gsize = min(GROUP_M, tiles_m - first_m);
    const int in_group = t - first_m * tiles_n;
    const int m0 = (first_m + in_group % gsize) * BM, n0 = (in_group / gsize) * BN;
    const int kb = blockIdx.z * a.ksplit;
    const int ke = min(a.K, kb + a.ksplit);
    const int nk = ke > kb ? (ke - kb + BK - 1) / BK : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *issued = 0;
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
    }
    if (warp == 0) {   // BN fp32 columns of tensor memory for the accumulator
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(tslot)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {   // producer: TMA copies of the operand tiles
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % STAGES;
            if (kt >= STAGES && !mbar_wait_bounded(empty + s, ((kt / STAGES) - 1) & 1, kWaitNs)) {
                *abort_flag = 1;
                break;
            }
            if (*abort_flag) break;
            mbar_arrive_expect(full + s, TILE_A + TILE_B);
            tma_load_2d(sA + s * TILE_A, &ta, kb + kt * BK, m0, full + s);
            tma_load_2d(sB + s * TILE_B, &tb, kb + kt * BK, n0, full + s);
            *issued = kt + 1;
        }
    } else if (warp == 1 && lane == 0) {   // MMA issuer
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % STAGES;
            if (!mbar_wait_bounded(full + s, (kt / STAGES) & 1, kWaitNs)) {
                *abort_flag = 1;
                break;
            }
            fence_after();
            const uint32_t a0 = s_addr(sA + s * TILE_A), b0 = s_addr(sB + s * TILE_B);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)   // 16 K-elements = 32 bytes along the swizzled row
                mma_bf16(tmem, desc_sw128(a0 + 32 * kk), desc_sw128(b0 + 32 * kk), idesc<BN>(), (kt | kk) ? 1u : 0u);
            mma_commit(empty + s);
        }
        mma_commit(done);
    }
    __syncwarp();
    // one decision for the whole CTA: tcgen05.ld below is a warp-collective instruction
    const bool waited = mbar_wait_bounded(done, 0, kWaitNs);
    const bool ok = __syncthreads_and(waited && !*abort_flag) != 0;
    fence_after();
    if (ok && nk > 0) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN && n0 + c0 < a.N; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr + uint32_t(c0)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < a.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n >= a.N) break;
                    float x = __uint_as_float(v[j]);
                    if (a.bias) x += a.bias[n];
                    if (a.relu) x = fmaxf(x, 0.f);
                    const size_t o = size_t(row) * a.ldc + n;
                    if (a.out_mode == 0)
                        static_cast<__nv_bfloat16*>(a.C)[o] = __float2bfloat16(x);
                    else if (a.out_mode == 1)
                        static_cast<float*>(a.C)[o] = x;
                    else
                        atomicAdd(static_cast<float*>(a.C) + o, x);
                }
            }
        }
    }
    if (!ok) {
        // a wait gave up: let the copies this CTA issued land before its shared memory goes
        if (threadIdx.x == 0) {
            const int n_iss = *issued;
            for (int kt = max(0, n_iss - STAGES); kt < n_iss; ++kt)
                mbar_wait_bounded(full + (kt % STAGES), (kt / STAGES) & 1, kWaitNs);
            if (a.status) atomicOr(a.status, PAT_STATUS_TC05);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D tensor map of a row-major [rows][K] bf16 matrix with row pitch ld, boxes of BK x box_rows
int make_map(CUtensorMap* m, const __nv_bfloat16* base, int rows, int K, int ld, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) {
        set_error("unet_gemm_tc05: cuTensorMapEncodeTiled is not available from the driver");
        return PAT_ECUDA;
    }
    const cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
    const cuuint64_t strides[1] = {cuuint64_t(ld) * 2};
    const cuuint32_t box[2] = {cuuint32_t(BK), cuuint32_t(box_rows)};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides,
                           box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("unet_gemm_tc05: cuTensorMapEncodeTiled failed (%d) for a %d x %d matrix, pitch %d", int(r), rows, K,
                  ld);
        return PAT_ECUDA;
    }
    return PAT_OK;
}

template <int BN>
int launch(cudaStream_t st, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, Args a) {
    static bool configured = false;
    if (!configured) {
        PAT_CUDA(cudaFuncSetAttribute(k_gemm_tc05<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(smem_bytes<BN>())));
        configured = true;
    }
    CUtensorMap ta, tb;
    int rc = make_map(&ta, A, a.M, a.K, lda, BM);
    if (rc == PAT_OK) rc = make_map(&tb, B, a.N, a.K, ldb, BN);
    if (rc != PAT_OK) return rc;
    const long long tiles = (long long)((a.M + BM - 1) / BM) * ((a.N + BN - 1) / BN);
    const int nz = (a.K + a.ksplit - 1) / a.ksplit;
    if (tiles > 2147483647LL || nz > 65535) {
        set_error("unet_gemm_tc05: too many tiles (M=%d N=%d, split %d)", a.M, a.N, nz);
        return PAT_EINVAL;
    }
    count_launch();
    k_gemm_tc05<BN><<<dim3(unsigned(tiles), 1, nz), THREADS, smem_bytes<BN>(), st>>>(ta, tb, a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "k_gemm_tc05");
}

}  // namespace tc05

bool unet_gemm_tc05_supported(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K) {
    // TMA: 16-byte aligned bases and pitches; at least one full K box; sizes within the map limits
    return M > 0 && N > 0 && K >= tc05::BK && lda % 8 == 0 && ldb % 8 == 0 && lda >= K && ldb >= K &&
           (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0 &&
           tc05::encoder() != nullptr;
}

int unet_gemm_tc05(cudaStream_t st, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N,
                   int K, const float* bias, int relu, void* C, int ldc, int out_mode, int splitk, int* d_status) {
    if (!unet_gemm_tc05_supported(A, lda, B, ldb, M, N, K)) {
        set_error("unet_gemm_tc05: unsupported operands (M=%d N=%d K=%d lda=%d ldb=%d)", M, N, K, lda, ldb);
        return PAT_EINVAL;
    }
    splitk = std::max(1, splitk);
    int ks = (K + splitk - 1) / splitk;
    ks = (ks + tc05::BK - 1) / tc05::BK * tc05::BK;   // split boundaries on whole K boxes
    tc05::Args a{M, N, K, ks, bias, relu, C, ldc, out_mode, d_status};
    // the wider N tile halves the A traffic per MMA, where N allows it and the product still has
    // at least two waves of tiles (fewer tiles would leave SMs idle)
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long wide_tiles = (long long)((M + tc05::BM - 1) / tc05::BM) * ((N + 255) / 256) *
                                 ((K + ks - 1) / ks);
    return (N >= 256 && wide_tiles >= 2LL * sms) ? tc05::launch<256>(st, A, lda, B, ldb, a)
                                                 : tc05::launch<128>(st, A, lda, B, ldb, a);
}

}  // namespace pat
