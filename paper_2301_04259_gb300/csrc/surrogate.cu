// surrogate.cu -- learned surrogate of the batched method (the paper has none).
//
// A small network maps 8 active-region parameters to 128 PCA coefficients of the residual
// spectrum F - F_q plus the log10 of its own expected RV error; queries outside the training
// ranges or with a predicted error above a threshold go back to the plain method.
//
//  * network: 8 -> 4 x 256 (GELU) -> 129, BF16 weights and activations as GEMM operands, FP32
//    accumulation, every product on the tensor cores (tc::gemm_tn), FP32 master weights and
//    Adam moments; one training step = 5 forward GEMMs, a loss kernel, 9 backward GEMMs (GELU'
//    fused into the epilogue of each dA GEMM), one bias-gradient kernel and one Adam kernel,
//    captured once into a CUDA graph and replayed for every batch.
//  * PCA: randomized SVD with power iterations (Halko, Martinsson & Tropp 2011) over the
//    mean-centred residuals, FP32 GEMMs on the SIMT cores, the small symmetric eigenproblems
//    (l x l) in FP64 on the host (cyclic Jacobi).
//  * reconstruction: residual = mean + coef . basis with both factors split into BF16 high and
//    low parts, [c_hi c_hi c_lo] . [V_hi V_lo V_hi]^T in one tensor-core GEMM (K = 3 x 128).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "tc_gemm.cuh"

using bf16 = __nv_bfloat16;

namespace soap {
namespace sur {

constexpr int kLayers = 5;

struct Layer {
    int out, in, out_pad;
    int64_t offW, offb;        // into the flat parameter vector [W1 | b1 | W2 | b2 | ...]
    bf16* Wb;                  // [out][in]
    bf16* WbT;                 // [in][out_pad] (zero columns past out)
};

struct LayerTable {
    int n;
    int out[kLayers], in[kLayers], out_pad[kLayers];
    int64_t offW[kLayers], offb[kLayers];
    bf16* Wb[kLayers];
    bf16* WbT[kLayers];
};

}  // namespace sur
}  // namespace soap

struct soap_surrogate {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_in = 8, hidden = 256, n_hidden = 4, n_coef = 128, n_out = 129, n_out_pad = 136;
    int batch = 0;
    int64_t n_params = 0;
    soap::sur::Layer L[soap::sur::kLayers];
    float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
    bf16* wbuf = nullptr;
    float lo[16] = {}, hi[16] = {};
    float* d_lohi = nullptr;                  // [2][n_in]
    float* coef_mean = nullptr;               // [n_coef] (standardisation of the targets)
    float* coef_std = nullptr;
    float* w_out = nullptr;                   // [n_out] loss weights of the current stage
    // training buffers (batch rows)
    bf16 *X0 = nullptr, *X0T = nullptr;
    float* Z[4] = {};
    bf16* A[4] = {};
    bf16* AT[4] = {};
    float* Y = nullptr;
    float* T = nullptr;
    bf16 *dY = nullptr, *dYT = nullptr;
    bf16* dZ[4] = {};
    bf16* dZT[4] = {};
    int* perm = nullptr;
    int64_t perm_cap = 0;
    int* d_step = nullptr;                    // [0] step within the epoch, [1] Adam step t
    float* d_lr = nullptr;
    double* d_loss = nullptr;
    unsigned int* flags = nullptr;
    // training graph (captured per (data pointers, steps per epoch, stage))
    cudaGraphExec_t graph = nullptr;
    std::vector<uint64_t> graph_key;
    // query buffers (chunk rows)
    int q_cap = 0;
    bf16 *qa = nullptr, *qb = nullptr;        // ping-pong activations [q_cap][256]
    float* qy = nullptr;                      // [q_cap][n_out_pad]
    bf16* qsplit = nullptr;                   // [q_cap][3 n_coef]
    bf16* qx0 = nullptr;                      // [q_cap][n_in] scaled query inputs
    // basis
    int64_t n_px = 0;
    float* mu = nullptr;                      // [n_px]
    bf16* vsplit = nullptr;                   // [n_px][3 n_coef]: V_hi | V_lo | V_hi
    soap_surrogate* error_net = nullptr;         // network whose output n_coef predicts the RV error
};

namespace soap {
namespace sur {

// ---------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float scale_in(float x, float lo, float hi) { return 2.0f * (x - lo) / (hi - lo) - 1.0f; }

// Batch rows from the shuffled data set: scaled inputs (BF16, row-major and transposed) and
// targets.  Step s of the epoch takes perm[s*B .. s*B + B).
__global__ void k_gather(const float* __restrict__ x, const float* __restrict__ t, const int* __restrict__ perm,
                         const int* __restrict__ d_step, int B, int n_in, int n_out, const float* __restrict__ lohi,
                         bf16* __restrict__ X0, bf16* __restrict__ X0T, float* __restrict__ T) {
    const int r = blockIdx.x;
    const int src = perm[(int64_t)d_step[0] * B + r];
    for (int i = threadIdx.x; i < n_in; i += blockDim.x) {
        const bf16 v = __float2bfloat16_rn(scale_in(x[(int64_t)src * n_in + i], lohi[i], lohi[n_in + i]));
        X0[(int64_t)r * n_in + i] = v;
        X0T[(int64_t)i * B + r] = v;
    }
    for (int j = threadIdx.x; j < n_out; j += blockDim.x) T[(int64_t)r * n_out + j] = t[(int64_t)src * n_out + j];
}

// L = sum_b sum_j w_j (y - t)^2 / B; dY = bf16(2 w_j (y - t) / B), row-major and transposed
// (zero in the padding columns j >= n_out).
__global__ void k_loss(const float* __restrict__ Y, int ldy, const float* __restrict__ T, int n_out, int n_pad, int B,
                       const float* __restrict__ w, bf16* __restrict__ dY, bf16* __restrict__ dYT, double* loss) {
    __shared__ double s_part[8];
    double part = 0;
    const int64_t n_el = (int64_t)B * n_pad;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n_pad), j = (int)(e % n_pad);
        float d = 0.0f;
        if (j < n_out) {
            const float res = Y[(int64_t)r * ldy + j] - T[(int64_t)r * n_out + j];
            part += (double)w[j] * (double)res * (double)res;
            d = 2.0f * w[j] * res / (float)B;
        }
        const bf16 v = __float2bfloat16_rn(d);
        dY[(int64_t)r * n_pad + j] = v;
        dYT[(int64_t)j * B + r] = v;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += s_part[k];
        atomicAdd(loss, s / B);
    }
}

// Bias gradients: db[o] = sum_b g[o][b] over the transposed BF16 gradients of one layer.
struct BiasJobs {
    const bf16* gT[kLayers];
    int rows[kLayers];
    float* db[kLayers];
};
__global__ void k_bias_grad(BiasJobs jobs, int B) {
    const int l = blockIdx.y;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= jobs.rows[l]) return;
    const bf16* row = jobs.gT[l] + (int64_t)warp * B;
    float s = 0.0f;
    for (int b = lane; b < B; b += 32) s += __bfloat162float(row[b]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) jobs.db[l][warp] = s;
}

// Adam (Kingma & Ba 2015, Algorithm 1) over the flat parameters, then the BF16 copies W and
// W^T.  mode 0 updates everything except the RV-error head (row n_coef of the last layer and its
// bias), mode 1 only the head, mode 2 everything.
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                       float* __restrict__ V, int64_t n, const int* __restrict__ d_step, const float* __restrict__ d_lr,
                       float b1, float b2, float eps, int mode, int64_t head_w0, int head_len, int64_t head_b,
                       LayerTable lt) {
    const int t = d_step[1] + 1;
    const float lr = d_lr[0];
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
            const bool head = (e >= head_w0 && e < head_w0 + head_len) || e == head_b;
        if (mode != 2 && head != (mode == 1)) continue;
        const float g = G[e];
        const float m = b1 * M[e] + (1.0f - b1) * g;
        const float v = b2 * V[e] + (1.0f - b2) * g * g;
        M[e] = m;
        V[e] = v;
        const float w = P[e] - lr * (m / c1) / (sqrtf(v / c2) + eps);
        P[e] = w;
        for (int l = 0; l < lt.n; l++) {
            const int64_t nw = (int64_t)lt.out[l] * lt.in[l];
            if (e >= lt.offW[l] && e < lt.offW[l] + nw) {
                const int64_t q = e - lt.offW[l];
                const int o = (int)(q / lt.in[l]), i = (int)(q % lt.in[l]);
                const bf16 wb = __float2bfloat16_rn(w);
                lt.Wb[l][q] = wb;
                lt.WbT[l][(int64_t)i * lt.out_pad[l] + o] = wb;
            }
        }
    }
}

__global__ void k_step_inc(int* d_step, int steps_per_epoch) {
    d_step[0] = (d_step[0] + 1) % steps_per_epoch;
    d_step[1] += 1;
}

// BF16 copies of all weights from the FP32 master (after set_params).
__global__ void k_cast_weights(const float* __restrict__ P, LayerTable lt) {
    const int l = blockIdx.y;
    const int64_t nw = (int64_t)lt.out[l] * lt.in[l];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nw; q += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(q / lt.in[l]), i = (int)(q % lt.in[l]);
        const bf16 wb = __float2bfloat16_rn(P[lt.offW[l] + q]);
        lt.Wb[l][q] = wb;
        lt.WbT[l][(int64_t)i * lt.out_pad[l] + o] = wb;
    }
}

// Query inputs: scaled BF16 rows and the in-range flag (every input inside [lo, hi]).
__global__ void k_query_in(const float* __restrict__ x, int64_t n, int n_in, const float* __restrict__ lohi,
                           bf16* __restrict__ X0, uint8_t* __restrict__ in_range) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        bool ok = true;
        for (int i = 0; i < n_in; i++) {
            const float v = x[r * n_in + i];
            ok = ok && v >= lohi[i] && v <= lohi[n_in + i];
            X0[r * n_in + i] = __float2bfloat16_rn(scale_in(v, lohi[i], lohi[n_in + i]));
        }
        if (in_range) in_range[r] = ok ? 1 : 0;
    }
}

// Network outputs -> coefficients in data units, predicted RV error (cm/s), acceptance, and the
// split-BF16 rows [c_hi c_hi c_lo] for the reconstruction GEMM.
__global__ void k_query_out(const float* __restrict__ Y, int ldy, const float* __restrict__ Yerr, int ldyerr,
                            int64_t n, int n_coef, const float* __restrict__ mean,
                            const float* __restrict__ sd, float thr_cms, uint8_t* __restrict__ accept,
                            float* __restrict__ pred_err, float* __restrict__ coef_out, bf16* __restrict__ split) {
    const int64_t n_el = n * (n_coef + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / (n_coef + 1);
        const int j = (int)(e % (n_coef + 1));
        const float y = Y[r * ldy + j];
        if (j == n_coef) {
            const float err = exp10f(Yerr[r * ldyerr + j]);
            if (pred_err) pred_err[r] = err;
            if (accept) accept[r] = (accept[r] && err <= thr_cms) ? 1 : 0;
            continue;
        }
        const float c = y * sd[j] + mean[j];
        if (coef_out) coef_out[r * n_coef + j] = c;
        const bf16 hi = __float2bfloat16_rn(c);
        const bf16 lo = __float2bfloat16_rn(c - __bfloat162float(hi));
        split[r * 3 * n_coef + j] = hi;
        split[r * 3 * n_coef + n_coef + j] = hi;
        split[r * 3 * n_coef + 2 * n_coef + j] = lo;
    }
}

// Split-BF16 coefficient rows [c_hi c_hi c_lo] from FP32 coefficients [n][k].
__global__ void k_split_rows(const float* __restrict__ coef, int64_t n, int k, bf16* __restrict__ split) {
    const int64_t n_el = n * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k;
        const int j = (int)(e % k);
        const float c = coef[e];
        const bf16 hi = __float2bfloat16_rn(c);
        const bf16 lo = __float2bfloat16_rn(c - __bfloat162float(hi));
        split[r * 3 * k + j] = hi;
        split[r * 3 * k + k + j] = hi;
        split[r * 3 * k + 2 * k + j] = lo;
    }
}

// Split-BF16 basis rows [V_hi V_lo V_hi] (per pixel) from the FP32 basis [k][p].
__global__ void k_basis_split(const float* __restrict__ basis, int k, int64_t p, bf16* __restrict__ out) {
    const int64_t n_el = (int64_t)k * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / p);
        const int64_t m = e % p;
        const float v = basis[e];
        const bf16 hi = __float2bfloat16_rn(v);
        const bf16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        out[m * 3 * k + c] = hi;
        out[m * 3 * k + k + c] = lo;
        out[m * 3 * k + 2 * k + c] = hi;
    }
}

// ---------------------------------------------------------------------------------------
// FP32 SIMT GEMM for the PCA: C = alpha * A B + beta * C with strided operands
// A(m, k) = A[m * sam + k * sak], B(k, n) = B[k * sbk + n * sbn].  64 x 64 tiles, 16-deep
// K slices in shared memory, 4 x 4 outputs per thread.
// ---------------------------------------------------------------------------------------
template <bool AK, bool BN_>
__global__ void __launch_bounds__(256)
k_sgemm(int M, int N, int64_t K, float alpha, const float* __restrict__ A, int64_t sam, int64_t sak,
        const float* __restrict__ B, int64_t sbk, int64_t sbn, float beta, float* __restrict__ C, int64_t ldc) {
    __shared__ float As[16][68];
    __shared__ float Bs[16][68];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int ty = tid / 16, tx = tid % 16;
    float acc[4][4] = {};
    for (int64_t k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int mm, kk;
            if (AK) { mm = tid / 4; kk = (tid % 4) * 4 + j; } else { kk = tid / 16; mm = (tid % 16) * 4 + j; }
            const int m = m0 + mm;
            const int64_t k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? A[(int64_t)m * sam + k * sak] : 0.0f;
            int nn, kb;
            if (BN_) { kb = tid / 16; nn = (tid % 16) * 4 + j; } else { nn = tid / 4; kb = (tid % 4) * 4 + j; }
            const int n = n0 + nn;
            const int64_t kq = k0 + kb;
            Bs[kb][nn] = (n < N && kq < K) ? B[kq * sbk + (int64_t)n * sbn] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; kk++) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) {
                float* c = C + (int64_t)m * ldc + n;
                *c = alpha * acc[i][j] + (beta != 0.0f ? beta * *c : 0.0f);
            }
        }
}

static soap_status sgemm(int M, int N, int64_t K, float alpha, const float* A, int64_t sam, int64_t sak,
                         const float* B, int64_t sbk, int64_t sbn, float beta, float* C, int64_t ldc, cudaStream_t st) {
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
    const bool ak = sak == 1, bn = sbn == 1;
    if (ak && bn) k_sgemm<true, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, ldc);
    else if (ak) k_sgemm<true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, ldc);
    else if (bn) k_sgemm<false, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, ldc);
    else k_sgemm<false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, ldc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error("sgemm launch failed: %s", cudaGetErrorString(e)); return SOAP_ECUDA; }
    return SOAP_OK;
}

__global__ void k_axpy(int64_t n, float alpha, const float* __restrict__ x, float* __restrict__ y) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = fmaf(alpha, x[e], y[e]);
}

// Network inputs of query parameters (soap_surrogate_encode): the region centre at the query's
// phase in the observer frame (the frame and angles of region_geometry, rigid rotation) and the
// parameters it does not fix.
__global__ void k_surrogate_encode(int64_t n, const float* __restrict__ q, float* __restrict__ x) {
    const float d2r = 0.017453292519943295f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float* p = q + 8 * i;
        float* o = x + 8 * i;
        float sl, cl, sL, cL, si, ci;
        sincosf(p[0] * d2r, &sl, &cl);
        sincosf((p[1] + 360.0f * p[4]) * d2r, &sL, &cL);
        sincosf(p[5] * d2r, &si, &ci);
        const float px = cl * sL, pc = cl * cL;
        o[0] = sl * si - pc * ci;
        o[1] = px;
        o[2] = p[2];
        o[3] = p[3];
        o[4] = sl * ci + pc * si;
        o[5] = p[6] * px;
        o[6] = p[6];
        o[7] = p[7];
    }
}

// column means of X [n][p] (FP64 accumulation)
__global__ void k_colmean(const float* __restrict__ X, int64_t n, int64_t p, float* __restrict__ mu) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < p; c += (int64_t)gridDim.x * blockDim.x) {
        double s = 0;
        for (int64_t r = 0; r < n; r++) s += X[r * p + c];
        mu[c] = (float)(s / (double)n);
    }
}

// C[m][j] -= u[m] * v[j]
__global__ void k_rank1_sub(float* __restrict__ C, int64_t ldc, int64_t M, int N, const float* __restrict__ u,
                            const float* __restrict__ v, bool u_ones) {
    const int64_t n_el = M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e / N;
        const int j = (int)(e % N);
        C[m * ldc + j] -= (u_ones ? 1.0f : u[m]) * v[j];
    }
}

// column sums of Q [n][l]
__global__ void k_colsum(const float* __restrict__ Q, int64_t n, int l, float* __restrict__ s) {
    const int j = blockIdx.x;
    double acc = 0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) acc += Q[r * l + j];
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) s[j] = (float)sh[0];
}

// ---------------------------------------------------------------------------------------
// host linear algebra (FP64): cyclic Jacobi eigen-decomposition of a symmetric matrix
// ---------------------------------------------------------------------------------------
static void jacobi_eig(int n, std::vector<double> a, std::vector<double>& w, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0, diag = 0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) (i == j ? diag : off) += a[(size_t)i * n + j] * a[(size_t)i * n + j];
        if (off <= 1e-30 * diag || off == 0) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                const double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; k++) {           // A <- A J (columns p, q)
                    const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {           // A <- J^T A (rows p, q)
                    const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {           // V <- V J
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; i++) w[i] = a[(size_t)i * n + i];
}

// Eigenpairs in decreasing order: returns permutation of columns.
static std::vector<int> order_desc(const std::vector<double>& w) {
    std::vector<int> idx(w.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return w[a] > w[b]; });
    return idx;
}

// Orthonormal basis of the columns of Y [n][l] (in place): Y <- Y U Lambda^{-1/2} from the
// eigen-decomposition of Y^T Y; directions with eigenvalue below 1e-12 of the largest are
// dropped (zero columns).
static soap_status orthonormalize(float* Y, int64_t n, int l, float* work_l2, float* tmp, cudaStream_t st) {
    SOAP_TRY(sgemm(l, l, n, 1.0f, Y, 1, l, Y, l, 1, 0.0f, work_l2, l, st));
    std::vector<float> g((size_t)l * l);
    SOAP_CUDA(cudaMemcpyAsync(g.data(), work_l2, g.size() * 4, cudaMemcpyDeviceToHost, st));
    SOAP_CUDA(cudaStreamSynchronize(st));
    std::vector<double> a(g.begin(), g.end()), w, V;
    for (int i = 0; i < l; i++)
        for (int j = 0; j < i; j++) a[(size_t)i * l + j] = a[(size_t)j * l + i] = 0.5 * (a[(size_t)i * l + j] + a[(size_t)j * l + i]);
    jacobi_eig(l, a, w, V);
    const double wmax = *std::max_element(w.begin(), w.end());
    std::vector<float> Wm((size_t)l * l, 0.0f);
    const std::vector<int> idx = order_desc(w);
    for (int c = 0; c < l; c++) {
        const int e = idx[c];
        if (!(w[e] > 1e-12 * wmax)) continue;
        const double f = 1.0 / std::sqrt(w[e]);
        for (int i = 0; i < l; i++) Wm[(size_t)i * l + c] = (float)(V[(size_t)i * l + e] * f);
    }
    SOAP_CUDA(cudaMemcpyAsync(work_l2, Wm.data(), Wm.size() * 4, cudaMemcpyHostToDevice, st));
    SOAP_TRY(sgemm((int)n, l, l, 1.0f, Y, l, 1, work_l2, l, 1, 0.0f, tmp, l, st));
    SOAP_CUDA(cudaMemcpyAsync(Y, tmp, (size_t)n * l * 4, cudaMemcpyDeviceToDevice, st));
    SOAP_CUDA(cudaStreamSynchronize(st));
    return SOAP_OK;
}

static int grid1(int64_t n, int threads = 256, int cap = 152 * 16) {
    int64_t g = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// ---------------------------------------------------------------------------------------
// network helpers
// ---------------------------------------------------------------------------------------
static LayerTable table(const soap_surrogate* s) {
    LayerTable lt{};
    lt.n = kLayers;
    for (int l = 0; l < kLayers; l++) {
        lt.out[l] = s->L[l].out; lt.in[l] = s->L[l].in; lt.out_pad[l] = s->L[l].out_pad;
        lt.offW[l] = s->L[l].offW; lt.offb[l] = s->L[l].offb;
        lt.Wb[l] = s->L[l].Wb; lt.WbT[l] = s->L[l].WbT;
    }
    return lt;
}

// Forward pass of B rows from X0 (BF16 [B][n_in]).  Training keeps z (FP32), a (BF16) and a^T;
// inference ping-pongs a between qa and qb.  Output y [B][n_out_pad] FP32.
static soap_status forward(soap_surrogate* s, const bf16* X0, int B, bool train, float* Yout) {
    const bf16* a = X0;
    int64_t lda = s->n_in;
    for (int l = 0; l < kLayers; l++) {
        const Layer& L = s->L[l];
        tc::Epilogue ep{};
        ep.bias = s->P + L.offb;
        if (l < kLayers - 1) {
            ep.flags = tc::EPI_BIAS | tc::EPI_GELU | tc::EPI_A16;
            if (train) {
                ep.flags |= tc::EPI_Z32 | tc::EPI_A16T;
                ep.c32 = s->Z[l]; ep.ldc32 = L.out;
                ep.c16 = s->A[l]; ep.ldc16 = L.out;
                ep.c16t = s->AT[l]; ep.ldc16t = B;
            } else {
                ep.c16 = (l % 2 == 0) ? s->qa : s->qb; ep.ldc16 = L.out;
            }
        } else {
            ep.flags = tc::EPI_BIAS | tc::EPI_A32;
            ep.c32 = Yout; ep.ldc32 = s->n_out_pad;
        }
        SOAP_TRY(tc::gemm_tn(a, lda, L.Wb, L.in, B, L.out, L.in, ep, s->stream, s->flags));
        a = train ? s->A[l] : ((l % 2 == 0) ? s->qa : s->qb);
        lda = L.out;
    }
    return SOAP_OK;
}

// Loss, backward pass and bias gradients for the batch in the training buffers; gradients into G.
static soap_status backward(soap_surrogate* s, int B) {
    const int blocks = grid1((int64_t)B * s->n_out_pad);
    k_loss<<<blocks, 256, 0, s->stream>>>(s->Y, s->n_out_pad, s->T, s->n_out, s->n_out_pad, B, s->w_out, s->dY,
                                          s->dYT, s->d_loss);
    const bf16* g = s->dY;        // gradient wrt the outputs of layer l (row-major)
    const bf16* gT = s->dYT;
    int64_t ldg = s->n_out_pad;
    BiasJobs bj{};
    for (int l = kLayers - 1; l >= 0; l--) {
        const Layer& L = s->L[l];
        // dW_l = g^T a_{l-1}:  A = g^T [out][B], B = a_{l-1}^T [in][B]
        tc::Epilogue ew{};
        ew.flags = tc::EPI_A32;
        ew.c32 = s->G + L.offW; ew.ldc32 = L.in;
        const bf16* aT = l == 0 ? s->X0T : s->AT[l - 1];
        SOAP_TRY(tc::gemm_tn(gT, B, aT, B, L.out, L.in, B, ew, s->stream, s->flags));
        bj.gT[l] = gT; bj.rows[l] = L.out; bj.db[l] = s->G + L.offb;
        if (l == 0) break;
        // dz_{l-1} = (g W_l) * GELU'(z_{l-1}):  A = g [B][out_pad], B = W_l^T [in][out_pad]
        tc::Epilogue ed{};
        ed.flags = tc::EPI_DGELU | tc::EPI_A16 | tc::EPI_A16T;
        ed.zin = s->Z[l - 1]; ed.ldzin = L.in;
        ed.c16 = s->dZ[l - 1]; ed.ldc16 = L.in;
        ed.c16t = s->dZT[l - 1]; ed.ldc16t = B;
        SOAP_TRY(tc::gemm_tn(g, ldg, L.WbT, L.out_pad, B, L.in, L.out_pad, ed, s->stream, s->flags));
        g = s->dZ[l - 1];
        gT = s->dZT[l - 1];
        ldg = L.in;
    }
    dim3 bg((unsigned)((std::max(s->hidden, s->n_out) * 32 + 255) / 256), kLayers);
    k_bias_grad<<<bg, 256, 0, s->stream>>>(bj, B);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error("kernel launch failed: %s", cudaGetErrorString(e)); return SOAP_ECUDA; }
    return SOAP_OK;
}

static soap_status alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) { *p = nullptr; set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e)); return SOAP_ENOMEM; }
    return SOAP_OK;
}

static soap_status ensure_query(soap_surrogate* s, int rows) {
    if (rows <= s->q_cap) return SOAP_OK;
    cudaStreamSynchronize(s->stream);
    cudaFree(s->qa); cudaFree(s->qb); cudaFree(s->qy); cudaFree(s->qsplit); cudaFree(s->qx0);
    s->qa = s->qb = nullptr; s->qy = nullptr; s->qsplit = nullptr; s->qx0 = nullptr; s->q_cap = 0;
    SOAP_TRY(alloc((void**)&s->qa, (size_t)rows * s->hidden * sizeof(bf16)));
    SOAP_TRY(alloc((void**)&s->qb, (size_t)rows * s->hidden * sizeof(bf16)));
    SOAP_TRY(alloc((void**)&s->qy, (size_t)rows * s->n_out_pad * sizeof(float)));
    SOAP_TRY(alloc((void**)&s->qsplit, (size_t)rows * 3 * s->n_coef * sizeof(bf16)));
    SOAP_TRY(alloc((void**)&s->qx0, (size_t)rows * s->n_in * sizeof(bf16)));
    s->q_cap = rows;
    return SOAP_OK;
}

// The error network (if any) runs on the same scaled inputs, on the main network's stream.
static soap_status error_net_forward(soap_surrogate* s, const bf16* X0, int m) {
    if (!s->error_net) return SOAP_OK;
    soap_surrogate* j = s->error_net;
    SOAP_TRY(ensure_query(j, s->q_cap));
    const cudaStream_t saved = j->stream;
    j->stream = s->stream;
    const soap_status st = forward(j, X0, m, false, j->qy);
    j->stream = saved;
    return st;
}

static soap_status check(soap_surrogate* s) {
    unsigned int h = 0, hj = 0;
    SOAP_CUDA(cudaMemcpyAsync(&h, s->flags, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    if (s->error_net) SOAP_CUDA(cudaMemcpyAsync(&hj, s->error_net->flags, sizeof(hj), cudaMemcpyDeviceToHost, s->stream));
    SOAP_CUDA(cudaStreamSynchronize(s->stream));
    h |= hj;
    if (h) {
        SOAP_CUDA(cudaMemsetAsync(s->flags, 0, sizeof(unsigned int), s->stream));
        if (s->error_net) SOAP_CUDA(cudaMemsetAsync(s->error_net->flags, 0, sizeof(unsigned int), s->stream));
        set_error("a tensor-core kernel gave up waiting (status 0x%x)", h);
        return SOAP_ETIMEOUT;
    }
    return SOAP_OK;
}

static void free_all(soap_surrogate* s) {
    if (s->graph) cudaGraphExecDestroy(s->graph);
    void* ptrs[] = {s->P, s->G, s->Mo, s->Vo, s->wbuf, s->d_lohi, s->coef_mean, s->coef_std, s->w_out, s->X0, s->X0T,
                    s->Y, s->T, s->dY, s->dYT, s->perm, s->d_step, s->d_lr, s->d_loss, s->flags, s->qa, s->qb,
                    s->qy, s->qsplit, s->qx0, s->mu, s->vsplit};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < 4; l++) {
        if (s->Z[l]) cudaFree(s->Z[l]);
        if (s->A[l]) cudaFree(s->A[l]);
        if (s->AT[l]) cudaFree(s->AT[l]);
        if (s->dZ[l]) cudaFree(s->dZ[l]);
        if (s->dZT[l]) cudaFree(s->dZT[l]);
    }
}

}  // namespace sur
}  // namespace soap

using namespace soap;
using namespace soap::sur;

extern "C" {

soap_status soap_surrogate_create(const soap_surrogate_desc* d, void* cuda_stream, soap_surrogate** out) {
    clear_error();
    if (!d || !out || !d->in_lo || !d->in_hi) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (d->n_in != 8 || d->hidden != 256 || d->n_hidden != 4 || d->n_coef != 128) {
        set_error("this build trains the 8 -> 4 x 256 -> 128 (+1) network only"); return SOAP_EINVAL;
    }
    if (d->batch < 128 || d->batch % 128 || d->batch > (1 << 20)) { set_error("batch must be a positive multiple of 128"); return SOAP_EINVAL; }
    for (int i = 0; i < d->n_in; i++)
        if (!(d->in_hi[i] > d->in_lo[i]) || !std::isfinite(d->in_lo[i]) || !std::isfinite(d->in_hi[i])) {
            set_error("input range %d invalid", i); return SOAP_EINVAL;
        }
    soap_surrogate* s = new (std::nothrow) soap_surrogate();
    if (!s) { set_error("out of host memory"); return SOAP_ENOMEM; }
    cudaGetDevice(&s->device);
    s->stream = (cudaStream_t)cuda_stream;
    s->batch = d->batch;
    for (int i = 0; i < s->n_in; i++) { s->lo[i] = d->in_lo[i]; s->hi[i] = d->in_hi[i]; }
    const int dims[kLayers + 1] = {s->n_in, s->hidden, s->hidden, s->hidden, s->hidden, s->n_out};
    int64_t off = 0, nwb = 0;
    for (int l = 0; l < kLayers; l++) {
        Layer& L = s->L[l];
        L.in = dims[l]; L.out = dims[l + 1]; L.out_pad = (L.out + 7) / 8 * 8;
        L.offW = off; off += (int64_t)L.out * L.in;
        L.offb = off; off += L.out;
        nwb += (int64_t)L.out * L.in + (int64_t)L.in * L.out_pad;
    }
    s->n_params = off;
    const int B = s->batch;
    soap_status st = SOAP_OK;
#define A_(p, bytes) if (st == SOAP_OK) st = alloc((void**)&(p), (bytes))
    A_(s->P, off * 4); A_(s->G, off * 4); A_(s->Mo, off * 4); A_(s->Vo, off * 4);
    A_(s->wbuf, nwb * sizeof(bf16));
    A_(s->d_lohi, 2 * s->n_in * 4);
    A_(s->coef_mean, s->n_coef * 4); A_(s->coef_std, s->n_coef * 4); A_(s->w_out, s->n_out * 4);
    A_(s->X0, (size_t)B * s->n_in * sizeof(bf16)); A_(s->X0T, (size_t)B * s->n_in * sizeof(bf16));
    for (int l = 0; l < 4; l++) {
        A_(s->Z[l], (size_t)B * s->hidden * 4);
        A_(s->A[l], (size_t)B * s->hidden * sizeof(bf16)); A_(s->AT[l], (size_t)B * s->hidden * sizeof(bf16));
        A_(s->dZ[l], (size_t)B * s->hidden * sizeof(bf16)); A_(s->dZT[l], (size_t)B * s->hidden * sizeof(bf16));
    }
    A_(s->Y, (size_t)B * s->n_out_pad * 4); A_(s->T, (size_t)B * s->n_out * 4);
    A_(s->dY, (size_t)B * s->n_out_pad * sizeof(bf16)); A_(s->dYT, (size_t)B * s->n_out_pad * sizeof(bf16));
    A_(s->d_step, 2 * sizeof(int)); A_(s->d_lr, sizeof(float)); A_(s->d_loss, sizeof(double));
    A_(s->flags, sizeof(unsigned int));
#undef A_
    if (st != SOAP_OK) { free_all(s); delete s; return st; }
    bf16* wp = s->wbuf;
    for (int l = 0; l < kLayers; l++) {
        Layer& L = s->L[l];
        L.Wb = wp; wp += (int64_t)L.out * L.in;
        L.WbT = wp; wp += (int64_t)L.in * L.out_pad;
    }
    float lohi[32];
    for (int i = 0; i < s->n_in; i++) { lohi[i] = s->lo[i]; lohi[s->n_in + i] = s->hi[i]; }
    std::vector<float> ones(s->n_coef, 1.0f), zeros(s->n_coef, 0.0f);
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    ok(cudaMemcpyAsync(s->d_lohi, lohi, 2 * s->n_in * 4, cudaMemcpyHostToDevice, s->stream));
    ok(cudaMemcpyAsync(s->coef_mean, zeros.data(), s->n_coef * 4, cudaMemcpyHostToDevice, s->stream));
    ok(cudaMemcpyAsync(s->coef_std, ones.data(), s->n_coef * 4, cudaMemcpyHostToDevice, s->stream));
    ok(cudaMemsetAsync(s->P, 0, off * 4, s->stream));
    ok(cudaMemsetAsync(s->wbuf, 0, nwb * sizeof(bf16), s->stream));
    ok(cudaMemsetAsync(s->Mo, 0, off * 4, s->stream));
    ok(cudaMemsetAsync(s->Vo, 0, off * 4, s->stream));
    ok(cudaMemsetAsync(s->d_step, 0, 2 * sizeof(int), s->stream));
    ok(cudaMemsetAsync(s->flags, 0, sizeof(unsigned int), s->stream));
    ok(cudaStreamSynchronize(s->stream));
    if (e != cudaSuccess) { set_error("initialisation failed: %s", cudaGetErrorString(e)); free_all(s); delete s; return SOAP_ECUDA; }
    *out = s;
    return SOAP_OK;
}

soap_status soap_surrogate_num_params(const soap_surrogate* s, int64_t* n) {
    clear_error();
    if (!s || !n) { set_error("NULL argument"); return SOAP_EINVAL; }
    *n = s->n_params;
    return SOAP_OK;
}

soap_status soap_surrogate_set_params(soap_surrogate* s, const float* flat) {
    clear_error();
    if (!s || !flat) { set_error("NULL argument"); return SOAP_EINVAL; }
    SOAP_CUDA(cudaMemcpyAsync(s->P, flat, s->n_params * 4, cudaMemcpyHostToDevice, s->stream));
    SOAP_CUDA(cudaMemsetAsync(s->Mo, 0, s->n_params * 4, s->stream));
    SOAP_CUDA(cudaMemsetAsync(s->Vo, 0, s->n_params * 4, s->stream));
    SOAP_CUDA(cudaMemsetAsync(s->d_step, 0, 2 * sizeof(int), s->stream));
    dim3 g(64, kLayers);
    k_cast_weights<<<g, 256, 0, s->stream>>>(s->P, table(s));
    SOAP_CUDA(cudaGetLastError());
    SOAP_CUDA(cudaStreamSynchronize(s->stream));
    return SOAP_OK;
}

soap_status soap_surrogate_get_params(soap_surrogate* s, float* flat) {
    clear_error();
    if (!s || !flat) { set_error("NULL argument"); return SOAP_EINVAL; }
    SOAP_CUDA(cudaMemcpyAsync(flat, s->P, s->n_params * 4, cudaMemcpyDeviceToHost, s->stream));
    SOAP_CUDA(cudaStreamSynchronize(s->stream));
    return SOAP_OK;
}

soap_status soap_surrogate_set_scaling(soap_surrogate* s, const float* coef_mean, const float* coef_std) {
    clear_error();
    if (!s || !coef_mean || !coef_std) { set_error("NULL argument"); return SOAP_EINVAL; }
    for (int j = 0; j < s->n_coef; j++)
        if (!(coef_std[j] > 0) || !std::isfinite(coef_mean[j])) { set_error("coef_std[%d] must be > 0", j); return SOAP_EINVAL; }
    SOAP_CUDA(cudaMemcpyAsync(s->coef_mean, coef_mean, s->n_coef * 4, cudaMemcpyHostToDevice, s->stream));
    SOAP_CUDA(cudaMemcpyAsync(s->coef_std, coef_std, s->n_coef * 4, cudaMemcpyHostToDevice, s->stream));
    SOAP_CUDA(cudaStreamSynchronize(s->stream));
    return SOAP_OK;
}

soap_status soap_surrogate_gradients(soap_surrogate* s, const float* x, const float* t, int32_t n,
                                     const float* w_out, double* loss, float* grads) {
    clear_error();
    if (!s || !x || !t || !w_out || !loss || !grads) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (n != s->batch) { set_error("n must equal the batch size (%d)", s->batch); return SOAP_EINVAL; }
    std::vector<int> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    if (s->perm_cap < n) {
        if (s->perm) cudaFree(s->perm);
        SOAP_TRY(alloc((void**)&s->perm, (size_t)n * sizeof(int)));
        s->perm_cap = n;
    }
    SOAP_CUDA(cudaMemcpyAsync(s->perm, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s->stream));
    SOAP_CUDA(cudaMemcpyAsync(s->w_out, w_out, s->n_out * 4, cudaMemcpyHostToDevice, s->stream));
    SOAP_CUDA(cudaMemsetAsync(s->d_step, 0, sizeof(int), s->stream));
    SOAP_CUDA(cudaMemsetAsync(s->d_loss, 0, sizeof(double), s->stream));
    k_gather<<<n, 32, 0, s->stream>>>(x, t, s->perm, s->d_step, n, s->n_in, s->n_out, s->d_lohi, s->X0, s->X0T, s->T);
    SOAP_CUDA(cudaGetLastError());
    SOAP_TRY(forward(s, s->X0, n, true, s->Y));
    SOAP_TRY(backward(s, n));
    SOAP_CUDA(cudaMemcpyAsync(loss, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SOAP_CUDA(cudaMemcpyAsync(grads, s->G, s->n_params * 4, cudaMemcpyDeviceToHost, s->stream));
    return check(s);
}

soap_status soap_surrogate_train(soap_surrogate* s, const float* x, const float* t, int64_t n, int32_t epochs,
                                 const float* lr_per_epoch, const float* w_out, int32_t stage, uint64_t seed,
                                 double* loss_per_epoch) {
    clear_error();
    if (!s || !x || !t || !lr_per_epoch || !w_out) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (stage < 0 || stage > 2) { set_error("stage must be 0 (all but the RV-error head), 1 (head) or 2 (all)"); return SOAP_EINVAL; }
    const int B = s->batch;
    const int64_t steps64 = n / B;
    if (steps64 < 1 || steps64 > (1 << 24)) { set_error("need at least one full batch of %d rows", B); return SOAP_EINVAL; }
    if (epochs < 0) { set_error("epochs < 0"); return SOAP_EINVAL; }
    const int steps = (int)steps64;
    if (s->perm_cap < n) {
        if (s->perm) cudaFree(s->perm);
        s->perm = nullptr; s->perm_cap = 0;
        SOAP_TRY(alloc((void**)&s->perm, (size_t)n * sizeof(int)));
        s->perm_cap = n;
    }
    SOAP_CUDA(cudaMemcpyAsync(s->w_out, w_out, s->n_out * 4, cudaMemcpyHostToDevice, s->stream));
    const Layer& last = s->L[kLayers - 1];
    const int64_t head_w0 = last.offW + (int64_t)s->n_coef * last.in;
    const int64_t head_b = last.offb + s->n_coef;
    // the graph of one step, keyed by what it bakes in
    std::vector<uint64_t> key = {(uint64_t)(uintptr_t)x, (uint64_t)(uintptr_t)t, (uint64_t)(uintptr_t)s->perm,
                                 (uint64_t)steps, (uint64_t)stage, (uint64_t)(uintptr_t)s->stream};
    if (!s->graph || s->graph_key != key) {
        if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
        cudaStream_t cap;
        SOAP_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        const cudaStream_t saved = s->stream;
        s->stream = cap;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        soap_status st = SOAP_OK;
        cudaGraph_t graph = nullptr;
        if (e == cudaSuccess) {
            k_gather<<<B, 32, 0, cap>>>(x, t, s->perm, s->d_step, B, s->n_in, s->n_out, s->d_lohi, s->X0, s->X0T, s->T);
            st = forward(s, s->X0, B, true, s->Y);
            if (st == SOAP_OK) st = backward(s, B);
            if (st == SOAP_OK) {
                k_adam<<<grid1(s->n_params), 256, 0, cap>>>(s->P, s->G, s->Mo, s->Vo, s->n_params, s->d_step, s->d_lr,
                                                             0.9f, 0.999f, 1e-8f, stage, head_w0, last.in, head_b, table(s));
                k_step_inc<<<1, 1, 0, cap>>>(s->d_step, steps);
            }
            const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
            if (e == cudaSuccess) e = e2;
        }
        s->stream = saved;
        if (st == SOAP_OK && e == cudaSuccess) e = cudaGraphInstantiate(&s->graph, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (st != SOAP_OK) { s->graph = nullptr; return st; }
        if (e != cudaSuccess) { s->graph = nullptr; set_error("training graph failed: %s", cudaGetErrorString(e)); return SOAP_ECUDA; }
        s->graph_key = key;
    }
    std::mt19937_64 rng(seed);
    std::vector<int> perm((size_t)n);
    SOAP_CUDA(cudaMemsetAsync(s->d_step, 0, sizeof(int), s->stream));      // step within epoch
    for (int ep = 0; ep < epochs; ep++) {
        std::iota(perm.begin(), perm.end(), 0);
        std::shuffle(perm.begin(), perm.end(), rng);
        SOAP_CUDA(cudaMemcpyAsync(s->perm, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s->stream));
        SOAP_CUDA(cudaMemcpyAsync(s->d_lr, &lr_per_epoch[ep], sizeof(float), cudaMemcpyHostToDevice, s->stream));
        SOAP_CUDA(cudaMemsetAsync(s->d_loss, 0, sizeof(double), s->stream));
        for (int k = 0; k < steps; k++) SOAP_CUDA(cudaGraphLaunch(s->graph, s->stream));
        double l = 0;
        SOAP_CUDA(cudaMemcpyAsync(&l, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        SOAP_CUDA(cudaStreamSynchronize(s->stream));       // perm and lr are reused next epoch
        if (loss_per_epoch) loss_per_epoch[ep] = l / steps;
    }
    return check(s);
}

soap_status soap_surrogate_predict(soap_surrogate* s, const float* x, int64_t n, float rv_err_max_cms,
                                   float* coef, float* pred_err_cms, uint8_t* accepted) {
    clear_error();
    if (!s || !x) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (n <= 0) return SOAP_OK;
    const int chunk = 65536;
    SOAP_TRY(ensure_query(s, (int)std::min<int64_t>(n, chunk)));
    bf16* X0 = s->qx0;
    soap_status st = SOAP_OK;
    for (int64_t r0 = 0; r0 < n && st == SOAP_OK; r0 += chunk) {
        const int m = (int)std::min<int64_t>(chunk, n - r0);
        k_query_in<<<grid1(m), 256, 0, s->stream>>>(x + r0 * s->n_in, m, s->n_in, s->d_lohi, X0,
                                                    accepted ? accepted + r0 : nullptr);
        st = forward(s, X0, m, false, s->qy);
        if (st == SOAP_OK) st = error_net_forward(s, X0, m);
        if (st != SOAP_OK) break;
        const float* ye = s->error_net ? s->error_net->qy : s->qy;
        k_query_out<<<grid1((int64_t)m * (s->n_coef + 1)), 256, 0, s->stream>>>(
            s->qy, s->n_out_pad, ye, s->n_out_pad, m, s->n_coef, s->coef_mean, s->coef_std, rv_err_max_cms,
            accepted ? accepted + r0 : nullptr, pred_err_cms ? pred_err_cms + r0 : nullptr,
            coef ? coef + r0 * s->n_coef : nullptr, s->qsplit);
    }
    SOAP_CUDA(cudaGetLastError());
    if (st != SOAP_OK) return st;
    return check(s);
}

soap_status soap_surrogate_set_error_net(soap_surrogate* s, soap_surrogate* error_net) {
    clear_error();
    if (!s) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (error_net == s) { set_error("a network cannot be its own error network"); return SOAP_EINVAL; }
    if (error_net) {
        for (int i = 0; i < s->n_in; i++)
            if (error_net->lo[i] != s->lo[i] || error_net->hi[i] != s->hi[i]) {
                set_error("the error network must use the same input ranges"); return SOAP_EINVAL;
            }
    }
    s->error_net = error_net;
    return SOAP_OK;
}

soap_status soap_surrogate_set_basis(soap_surrogate* s, const float* mean, const float* basis, int64_t n_px) {
    clear_error();
    if (!s || !mean || !basis || n_px < 1) { set_error("NULL argument or n_px < 1"); return SOAP_EINVAL; }
    if (s->mu) cudaFree(s->mu);
    if (s->vsplit) cudaFree(s->vsplit);
    s->mu = nullptr; s->vsplit = nullptr;
    SOAP_TRY(alloc((void**)&s->mu, (size_t)n_px * 4));
    SOAP_TRY(alloc((void**)&s->vsplit, (size_t)n_px * 3 * s->n_coef * sizeof(bf16)));
    s->n_px = n_px;
    SOAP_CUDA(cudaMemcpyAsync(s->mu, mean, (size_t)n_px * 4, cudaMemcpyDeviceToDevice, s->stream));
    k_basis_split<<<grid1((int64_t)s->n_coef * n_px), 256, 0, s->stream>>>(basis, s->n_coef, n_px, s->vsplit);
    SOAP_CUDA(cudaGetLastError());
    SOAP_CUDA(cudaStreamSynchronize(s->stream));
    return SOAP_OK;
}

soap_status soap_surrogate_query(soap_surrogate* s, const float* x, int64_t n, float rv_err_max_cms, float* out,
                                 float* pred_err_cms, uint8_t* accepted) {
    clear_error();
    if (!s || !x || !out || !accepted) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (!s->vsplit) { set_error("no basis set (soap_surrogate_set_basis)"); return SOAP_ESTATE; }
    if (n <= 0) return SOAP_OK;
    const int chunk = 65536;
    SOAP_TRY(ensure_query(s, (int)std::min<int64_t>(n, chunk)));
    bf16* X0 = s->qx0;
    soap_status st = SOAP_OK;
    for (int64_t r0 = 0; r0 < n && st == SOAP_OK; r0 += chunk) {
        const int m = (int)std::min<int64_t>(chunk, n - r0);
        k_query_in<<<grid1(m), 256, 0, s->stream>>>(x + r0 * s->n_in, m, s->n_in, s->d_lohi, X0, accepted + r0);
        st = forward(s, X0, m, false, s->qy);
        if (st == SOAP_OK) st = error_net_forward(s, X0, m);
        if (st != SOAP_OK) break;
        const float* ye = s->error_net ? s->error_net->qy : s->qy;
        k_query_out<<<grid1((int64_t)m * (s->n_coef + 1)), 256, 0, s->stream>>>(
            s->qy, s->n_out_pad, ye, s->n_out_pad, m, s->n_coef, s->coef_mean, s->coef_std, rv_err_max_cms,
            accepted + r0, pred_err_cms ? pred_err_cms + r0 : nullptr, nullptr, s->qsplit);
        tc::Epilogue ep{};
        ep.flags = tc::EPI_BIAS | tc::EPI_A32;
        ep.bias = s->mu;
        ep.c32 = out + r0 * s->n_px;
        ep.ldc32 = s->n_px;
        st = tc::gemm_tn(s->qsplit, 3 * s->n_coef, s->vsplit, 3 * s->n_coef, m, (int)s->n_px, 3 * s->n_coef, ep,
                         s->stream, s->flags);
    }
    if (st != SOAP_OK) return st;
    return check(s);
}

soap_status soap_surrogate_reconstruct(soap_surrogate* s, const float* coef, int64_t n, float* out) {
    clear_error();
    if (!s || !coef || !out) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (!s->vsplit) { set_error("no basis set (soap_surrogate_set_basis)"); return SOAP_ESTATE; }
    const int chunk = 65536;
    SOAP_TRY(ensure_query(s, (int)std::min<int64_t>(std::max<int64_t>(n, 1), chunk)));
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int m = (int)std::min<int64_t>(chunk, n - r0);
        k_split_rows<<<grid1((int64_t)m * s->n_coef), 256, 0, s->stream>>>(coef + r0 * s->n_coef, m, s->n_coef,
                                                                           s->qsplit);
        tc::Epilogue ep{};
        ep.flags = tc::EPI_BIAS | tc::EPI_A32;
        ep.bias = s->mu;
        ep.c32 = out + r0 * s->n_px;
        ep.ldc32 = s->n_px;
        SOAP_TRY(tc::gemm_tn(s->qsplit, 3 * s->n_coef, s->vsplit, 3 * s->n_coef, m, (int)s->n_px, 3 * s->n_coef,
                             ep, s->stream, s->flags));
    }
    return check(s);
}

void soap_surrogate_free(soap_surrogate* s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    free_all(s);
    delete s;
}

soap_status soap_surrogate_encode(const float* params, int64_t n, float* x, void* cuda_stream) {
    clear_error();
    if (n < 0) { set_error("invalid argument"); return SOAP_EINVAL; }
    if (n == 0) return SOAP_OK;
    if (!params || !x) { set_error("NULL argument"); return SOAP_EINVAL; }
    k_surrogate_encode<<<grid1(n), 256, 0, (cudaStream_t)cuda_stream>>>(n, params, x);
    SOAP_CUDA(cudaGetLastError());
    return SOAP_OK;
}

soap_status soap_axpy_f32(int64_t n, float alpha, const float* x, float* y, void* cuda_stream) {
    clear_error();
    if (!x || !y || n < 0) { set_error("invalid argument"); return SOAP_EINVAL; }
    if (n == 0) return SOAP_OK;
    k_axpy<<<grid1(n), 256, 0, (cudaStream_t)cuda_stream>>>(n, alpha, x, y);
    SOAP_CUDA(cudaGetLastError());
    return SOAP_OK;
}

// ---------------------------------------------------------------------------------------
// PCA
// ---------------------------------------------------------------------------------------
soap_status soap_pca_fit(const float* X, int64_t n, int64_t p, const float* omega, int32_t l, int32_t k,
                         int32_t n_power, float* mean, float* basis, double* sv, void* cuda_stream) {
    clear_error();
    if (!X || !omega || !mean || !basis) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (n < 2 || p < 1 || l < 1 || k < 1 || k > l || l > 512 || l > p || n_power < 0 || n_power > 10) {
        set_error("need n >= 2, 1 <= k <= l <= min(512, p), 0 <= n_power <= 10"); return SOAP_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    float *Y = nullptr, *Z = nullptr, *tmp = nullptr, *w2 = nullptr, *vecl = nullptr, *tmpz = nullptr;
    soap_status rc = SOAP_OK;
    auto A = [&](float** p_, size_t bytes) { if (rc == SOAP_OK) rc = alloc((void**)p_, bytes); };
    A(&Y, (size_t)n * l * 4); A(&tmp, (size_t)n * l * 4); A(&Z, (size_t)p * l * 4); A(&tmpz, (size_t)p * l * 4);
    A(&w2, (size_t)l * l * 4); A(&vecl, (size_t)l * 4);
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        for (float* q : {Y, Z, tmp, w2, vecl, tmpz}) if (q) cudaFree(q);
    };
    if (rc != SOAP_OK) { cleanup(); return rc; }
    auto run = [&]() -> soap_status {
        k_colmean<<<grid1(p), 256, 0, st>>>(X, n, p, mean);
        // Y = (X - 1 mu^T) Omega
        SOAP_TRY(sgemm((int)n, l, p, 1.0f, X, p, 1, omega, l, 1, 0.0f, Y, l, st));
        SOAP_TRY(sgemm(1, l, p, 1.0f, mean, 0, 1, omega, l, 1, 0.0f, vecl, l, st));
        k_rank1_sub<<<grid1(n * l), 256, 0, st>>>(Y, l, n, l, nullptr, vecl, true);
        for (int it = 0; it <= n_power; it++) {
            SOAP_TRY(orthonormalize(Y, n, l, w2, tmp, st));
            // Z = (X - 1 mu^T)^T Q = X^T Q - mu (1^T Q)
            SOAP_TRY(sgemm((int)p, l, n, 1.0f, X, 1, p, Y, l, 1, 0.0f, Z, l, st));
            k_colsum<<<l, 256, 0, st>>>(Y, n, l, vecl);
            k_rank1_sub<<<grid1(p * l), 256, 0, st>>>(Z, l, p, l, mean, vecl, false);
            if (it == n_power) break;
            SOAP_TRY(orthonormalize(Z, p, l, w2, tmpz, st));
            // Y = (X - 1 mu^T) Z
            SOAP_TRY(sgemm((int)n, l, p, 1.0f, X, p, 1, Z, l, 1, 0.0f, Y, l, st));
            SOAP_TRY(sgemm(1, l, p, 1.0f, mean, 0, 1, Z, l, 1, 0.0f, vecl, l, st));
            k_rank1_sub<<<grid1(n * l), 256, 0, st>>>(Y, l, n, l, nullptr, vecl, true);
        }
        // Z = B^T (p x l) with B = Q^T Xc; C = B B^T = Z^T Z; Xc ~ Q U S V^T with V = Z U S^-1
        SOAP_TRY(sgemm(l, l, p, 1.0f, Z, 1, l, Z, l, 1, 0.0f, w2, l, st));
        std::vector<float> g((size_t)l * l);
        SOAP_CUDA(cudaMemcpyAsync(g.data(), w2, g.size() * 4, cudaMemcpyDeviceToHost, st));
        SOAP_CUDA(cudaStreamSynchronize(st));
        std::vector<double> a(g.begin(), g.end()), w, V;
        for (int i = 0; i < l; i++)
            for (int j = 0; j < i; j++) a[(size_t)i * l + j] = a[(size_t)j * l + i] = 0.5 * (a[(size_t)i * l + j] + a[(size_t)j * l + i]);
        jacobi_eig(l, a, w, V);
        const std::vector<int> idx = order_desc(w);
        std::vector<float> Wm((size_t)l * k, 0.0f);
        for (int c = 0; c < k; c++) {
            const int e = idx[c];
            const double lam = std::max(w[e], 0.0);
            if (sv) sv[c] = std::sqrt(lam);
            const double f = lam > 0 ? 1.0 / std::sqrt(lam) : 0.0;
            for (int i = 0; i < l; i++) Wm[(size_t)i * k + c] = (float)(V[(size_t)i * l + e] * f);
        }
        SOAP_CUDA(cudaMemcpyAsync(w2, Wm.data(), Wm.size() * 4, cudaMemcpyHostToDevice, st));
        // basis [k][p] = (Z W)^T:  basis[c][m] = sum_i Z[m][i] W[i][c]
        SOAP_TRY(sgemm(k, (int)p, l, 1.0f, w2, 1, k, Z, 1, l, 0.0f, basis, p, st));
        SOAP_CUDA(cudaStreamSynchronize(st));
        return SOAP_OK;
    };
    rc = run();
    cleanup();
    return rc;
}

soap_status soap_pca_project(const float* X, int64_t n, int64_t p, const float* mean, const float* basis, int32_t k,
                             float* coef, void* cuda_stream) {
    clear_error();
    if (!X || !mean || !basis || !coef || n < 1 || p < 1 || k < 1) { set_error("invalid argument"); return SOAP_EINVAL; }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    float* v = nullptr;
    SOAP_TRY(alloc((void**)&v, (size_t)k * 4));
    // coef = X basis^T - 1 (mu . basis^T)
    soap_status rc = sgemm((int)n, k, p, 1.0f, X, p, 1, basis, 1, p, 0.0f, coef, k, st);
    if (rc == SOAP_OK) rc = sgemm(1, k, p, 1.0f, mean, 0, 1, basis, 1, p, 0.0f, v, k, st);
    if (rc == SOAP_OK) k_rank1_sub<<<grid1(n * k), 256, 0, st>>>(coef, k, n, k, nullptr, v, true);
    cudaStreamSynchronize(st);
    cudaFree(v);
    if (rc == SOAP_OK && cudaGetLastError() != cudaSuccess) { set_error("PCA projection failed"); rc = SOAP_ECUDA; }
    return rc;
}

}  // extern "C"
