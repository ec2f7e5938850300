// tc_gemm.cuh -- BF16 GEMM on the fifth-generation tensor cores (tcgen05) of sm_103a.
//
//   C[m][n] = epilogue( sum_k A[m][k] * B[n][k] )        ("TN": both operands K-contiguous)
//
// One CTA computes a 128 x BN tile.  Warp 0 streams 128 x 64 (A) and BN x 64 (B) BF16 tiles
// into shared memory with TMA (128-byte swizzle) through a ring of mbarriers (2 to 4 stages);
// warp 1 owns the tensor-memory accumulator (128 lanes x BN FP32 columns) and issues
// tcgen05.mma (M = 128, N = BN, K = 16 per instruction) from one thread; warps 2..5 read the
// accumulator back with tcgen05.ld (one row per thread) and apply the epilogue.
//
// Every wait is bounded (about a second of clock cycles); a wait that gives up sets
// kFlagTimeout in the caller's status word, the CTA stops issuing work, waits (bounded) for
// its own copies and MMAs in flight, frees its tensor memory and exits.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "soap_internal.cuh"

namespace soap {
namespace tc {

constexpr int BM = 128;        // rows per CTA (TMEM lanes)
constexpr int BK = 64;         // K elements per stage: one 128-byte swizzle atom of BF16
constexpr int kThreads = 192;
// Pipeline depth per tile width: two CTAs fit on an SM (shared memory and 512 TMEM columns), so
// one CTA's loads and MMAs overlap the other's epilogue.
template <int BN> struct Stages { static constexpr int value = BN >= 256 ? 2 : (BN >= 128 ? 3 : 4); };

// Epilogue: z = acc (+ bias[n]); a = GELU(z) when EPI_GELU, a = z * GELU'(zin[m][n]) when
// EPI_DGELU, else a = z.  Outputs (any subset): c32 <- z (EPI_Z32) or a (EPI_A32), c16 <- bf16(a),
// c16t[n][m] <- bf16(a) (transposed copy).
enum Epi : int {
    EPI_BIAS = 1, EPI_GELU = 2, EPI_DGELU = 4, EPI_Z32 = 8, EPI_A32 = 16, EPI_A16 = 32, EPI_A16T = 64
};

struct Epilogue {
    int flags;
    const float* bias;
    const float* zin; int64_t ldzin;
    float* c32; int64_t ldc32;
    __nv_bfloat16* c16; int64_t ldc16;
    __nv_bfloat16* c16t; int64_t ldc16t;
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    // d/dz [z Phi(z)] = Phi(z) + z phi(z)
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of parity `parity` to complete; false (and the flag) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned int* flags) {
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) {
            atomicOr(flags, kFlagTimeout);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 bytes
// apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                          // version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4)                       // D format FP32
           | (1u << 7)                     // A format BF16
           | (1u << 10)                    // B format BF16
           | ((uint32_t)(n >> 3) << 17)    // N / 8
           | ((uint32_t)(BM >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

template <int BN>
struct Smem {
    static constexpr int STAGES = Stages<BN>::value;
    static constexpr int kA = BM * BK * 2;          // bytes per stage
    static constexpr int kB = BN * BK * 2;
    static constexpr int kStage = kA + kB;
    static constexpr int kTile = 32 * 33 * 4;       // per epilogue warp: 32 x 32 floats, padded rows
    static_assert(4 * kTile <= STAGES * kStage, "epilogue tiles reuse the operand ring");
    static constexpr int kBytes = STAGES * kStage + 1024 /* alignment slack */ + 256 /* barriers */;
};

// Row-major store of a warp's 32 x 32 block through its shared tile: lane r holds row r's 32
// values; after the transpose, lane j writes column j of each row in turn, so every store
// instruction covers 32 consecutive elements of one row.
template <typename T>
__device__ __forceinline__ void store_rows(float (*tile)[33], const float (&v)[32], int lane, T* base, int64_t ld,
                                           int m_first, int M, int n_first, int N) {
#pragma unroll
    for (int i = 0; i < 32; i++) tile[lane][i] = v[i];
    __syncwarp();
    const int n = n_first + lane;
    if (n < N) {
#pragma unroll 4
        for (int r = 0; r < 32; r++) {
            const int m = m_first + r;
            if (m >= M) break;
            const float x = tile[r][lane];
            if constexpr (sizeof(T) == 4) base[(int64_t)m * ld + n] = x;
            else base[(int64_t)m * ld + n] = __float2bfloat16_rn(x);
        }
    }
    __syncwarp();
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 2)
k_gemm_tn(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, int M, int N,
          int K, Epilogue ep, unsigned int* flags) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05 N for M = 128");
    constexpr int STAGES = Smem<BN>::STAGES;
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned operand ring (the swizzle atom), barriers after it
    unsigned char* ring = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t* full = reinterpret_cast<uint64_t*>(ring + STAGES * Smem<BN>::kStage);
    uint64_t* empty = full + STAGES;
    uint64_t* accum = empty + STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    // epilogue tiles: the operand ring, free once the accumulator is complete (every copy has
    // been consumed by an MMA that has finished)
    float (*tiles)[32][33] = reinterpret_cast<float (*)[32][33]>(ring);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
    const int n_kb = (K + BK - 1) / BK;
    constexpr uint32_t kCols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(kCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer
        int armed = 0;
        bool ok = true;
        for (int kb = 0; kb < n_kb && ok; kb++) {
            const int s = kb % STAGES;
            const uint32_t ph = (kb / STAGES) & 1;
            if (!mbar_wait(&empty[s], ph ^ 1, flags)) { ok = false; break; }
            unsigned char* a = ring + s * Smem<BN>::kStage;
            mbar_expect_tx(&full[s], Smem<BN>::kStage);
            tma_load_2d(a, &map_a, kb * BK, m0, &full[s]);
            tma_load_2d(a + Smem<BN>::kA, &map_b, kb * BK, n0, &full[s]);
            armed = kb + 1;
        }
        // the last copies issued must land before the CTA may exit
        for (int kb = armed - 1; kb >= 0 && kb >= armed - STAGES; kb--)
            mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, flags);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BN);
        bool ok = true;
        int issued = 0;
        for (int kb = 0; kb < n_kb; kb++) {
            const int s = kb % STAGES;
            if (!mbar_wait(&full[s], (kb / STAGES) & 1, flags)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a = smem_u32(ring + s * Smem<BN>::kStage);
            const uint32_t b = a + Smem<BN>::kA;
#pragma unroll
            for (int k = 0; k < BK / 16; k++)
                mma_bf16(tmem, sdesc(a + k * 32), sdesc(b + k * 32), idesc, (kb | k) != 0);
            mma_commit(&empty[s]);
            issued = kb + 1;
        }
        (void)ok;
        mma_commit(accum);          // arrives once every MMA issued above has completed
        mbar_wait(accum, 0, flags); // (bounded) before the tensor memory can be released
        (void)issued;
    } else if (warp >= 2) {
        // epilogue: TMEM lanes 32*(warp % 4) .. +31
        const int lane_base = 32 * (warp & 3);
        const int m = m0 + lane_base + lane;
        // warp-uniform decision: tcgen05.ld is a warp-wide (.sync.aligned) instruction
        const bool done = __all_sync(0xffffffffu, mbar_wait(accum, 0, flags));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (done) {
            float (*tile)[33] = tiles[warp - 2];
            const int m_first = m0 + lane_base;
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
                if (n0 + c >= N) break;
                float v[32];
                tmem_ld32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)c, v);
                float a[32];
                if (ep.flags & EPI_DGELU) {
                    // GELU'(z_in) at this block: staged through the tile so the reads are by row
                    float zi[32];
#pragma unroll 4
                    for (int r = 0; r < 32; r++) {
                        const int mm = m_first + r, nn = n0 + c + lane;
                        tile[r][lane] = (mm < M && nn < N) ? ep.zin[(int64_t)mm * ep.ldzin + nn] : 0.0f;
                    }
                    __syncwarp();
#pragma unroll
                    for (int i = 0; i < 32; i++) zi[i] = tile[lane][i];
                    __syncwarp();
#pragma unroll
                    for (int i = 0; i < 32; i++) {
                        const float z = (ep.flags & EPI_BIAS) && n0 + c + i < N ? v[i] + ep.bias[n0 + c + i] : v[i];
                        v[i] = z;
                        a[i] = z * gelu_grad(zi[i]);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; i++) {
                        const int n = n0 + c + i;
                        const float z = (ep.flags & EPI_BIAS) && n < N ? v[i] + ep.bias[n] : v[i];
                        v[i] = z;
                        a[i] = (ep.flags & EPI_GELU) ? gelu(z) : z;
                    }
                }
                if (ep.flags & EPI_Z32) store_rows(tile, v, lane, ep.c32, ep.ldc32, m_first, M, n0 + c, N);
                if (ep.flags & EPI_A32) store_rows(tile, a, lane, ep.c32, ep.ldc32, m_first, M, n0 + c, N);
                if (ep.flags & EPI_A16) store_rows(tile, a, lane, ep.c16, ep.ldc16, m_first, M, n0 + c, N);
                if ((ep.flags & EPI_A16T) && m < M) {
#pragma unroll
                    for (int i = 0; i < 32; i++) {
                        const int n = n0 + c + i;
                        if (n < N) ep.c16t[(int64_t)n * ep.ldc16t + m] = __float2bfloat16_rn(a[i]);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

// Tiled tensor map without swizzle (BF16 elements unless dt says otherwise): dims[0] innermost
// (elements), strides in bytes of dims 1 .. rank-1, box in elements.  Zero fill outside the tensor.
soap_status encode_map(CUtensorMap* map, int rank, const void* base, const uint64_t* dims,
                       const uint64_t* strides, const uint32_t* box,
                       CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);

// C = epilogue(A B^T): A [M][K] (row stride lda), B [N][K] (row stride ldb), BF16, device, with
// 16-byte aligned bases and strides that are multiples of 8 elements.  Asynchronous on `st`.
soap_status gemm_tn(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int M, int N,
                    int K, const Epilogue& ep, cudaStream_t st, unsigned int* flags);

}  // namespace tc
}  // namespace soap
