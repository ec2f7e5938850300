// tc_gemm.cu -- host side of the tcgen05 BF16 GEMM: tensor maps, tile choice, launch.
#include <cudaTypedefs.h>

#include <mutex>

#include "tc_gemm.cuh"

namespace soap {
namespace tc {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Row-major BF16 matrix [rows][cols] with row stride ld (elements), boxes of box_rows x 64.
static soap_status make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                            int box_rows) {
    auto fn = encode_fn();
    if (!fn) { set_error("cuTensorMapEncodeTiled is not available from the driver"); return SOAP_ECUDA; }
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * 2) % 16 || ld < cols) {
        set_error("GEMM operand needs a 16-byte aligned base and a row stride that is a multiple of 8 elements");
        return SOAP_EINVAL;
    }
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled failed (%d)", (int)r); return SOAP_ECUDA; }
    return SOAP_OK;
}

soap_status encode_map(CUtensorMap* map, int rank, const void* base, const uint64_t* dims,
                       const uint64_t* strides, const uint32_t* box, CUtensorMapDataType dt) {
    auto fn = encode_fn();
    if (!fn) { set_error("cuTensorMapEncodeTiled is not available from the driver"); return SOAP_ECUDA; }
    if (rank < 1 || rank > 5 || (reinterpret_cast<uintptr_t>(base) & 15)) {
        set_error("tensor map: rank 1..5 and a 16-byte aligned base needed");
        return SOAP_EINVAL;
    }
    cuuint64_t d[5];
    cuuint64_t st[4];
    cuuint32_t bx[5], estr[5];
    for (int i = 0; i < rank; i++) {
        d[i] = (cuuint64_t)dims[i];
        bx[i] = (cuuint32_t)box[i];
        estr[i] = 1;
        if (i + 1 < rank) st[i] = (cuuint64_t)strides[i];
    }
    CUresult r = fn(map, dt, (cuuint32_t)rank, const_cast<void*>(base), d, st, bx, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled failed (%d)", (int)r); return SOAP_ECUDA; }
    return SOAP_OK;
}

template <int BN>
static soap_status launch(const CUtensorMap& ma, const CUtensorMap& mb, int M, int N, int K, const Epilogue& ep,
                          cudaStream_t st, unsigned int* flags) {
    static bool configured = false;     // per instantiation; attribute set is idempotent
    if (!configured) {
        SOAP_CUDA(cudaFuncSetAttribute(k_gemm_tn<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Smem<BN>::kBytes));
        configured = true;
    }
    dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
    k_gemm_tn<BN><<<grid, kThreads, Smem<BN>::kBytes, st>>>(ma, mb, M, N, K, ep, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error("GEMM launch failed: %s", cudaGetErrorString(e)); return SOAP_ECUDA; }
    return SOAP_OK;
}

soap_status gemm_tn(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int M, int N,
                    int K, const Epilogue& ep, cudaStream_t st, unsigned int* flags) {
    if (M <= 0 || N <= 0 || K <= 0) { set_error("GEMM sizes must be positive"); return SOAP_EINVAL; }
    const int BN = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
    CUtensorMap ma, mb;
    SOAP_TRY(make_map(&ma, A, M, K, lda, BM));
    SOAP_TRY(make_map(&mb, B, N, K, ldb, BN));
    if (BN == 64) return launch<64>(ma, mb, M, N, K, ep, st, flags);
    if (BN == 128) return launch<128>(ma, mb, M, N, K, ep, st, flags);
    return launch<256>(ma, mb, M, N, K, ep, st, flags);
}

}  // namespace tc
}  // namespace soap

using namespace soap;

// Status word of the context-free GEMM entry point.
static __device__ unsigned int g_gemm_flags;

extern "C" soap_status soap_gemm_bf16_tn(int32_t M, int32_t N, int32_t K, const void* A, int64_t lda,
                                         const void* B, int64_t ldb, const float* bias, int32_t activation,
                                         float* C, int64_t ldc, void* cuda_stream) {
    clear_error();
    if (!A || !B || !C) { set_error("NULL operand"); return SOAP_EINVAL; }
    if (activation != 0 && activation != 1) { set_error("activation must be 0 (none) or 1 (GELU)"); return SOAP_EINVAL; }
    if (ldc < N) { set_error("ldc < N"); return SOAP_EINVAL; }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned int* flags = nullptr;
    SOAP_CUDA(cudaGetSymbolAddress((void**)&flags, g_gemm_flags));
    SOAP_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned int), st));
    tc::Epilogue ep{};
    ep.flags = tc::EPI_A32 | (bias ? tc::EPI_BIAS : 0) | (activation ? tc::EPI_GELU : 0);
    ep.bias = bias;
    ep.c32 = C;
    ep.ldc32 = ldc;
    SOAP_TRY(tc::gemm_tn((const __nv_bfloat16*)A, lda, (const __nv_bfloat16*)B, ldb, M, N, K, ep, st, flags));
    unsigned int h = 0;
    SOAP_CUDA(cudaMemcpyAsync(&h, flags, sizeof(h), cudaMemcpyDeviceToHost, st));
    SOAP_CUDA(cudaStreamSynchronize(st));
    if (h) { set_error("GEMM kernel gave up waiting (status 0x%x)", h); return SOAP_ETIMEOUT; }
    return SOAP_OK;
}
