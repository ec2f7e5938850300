// geometry.cu -- G1: disk-cell geometry (Sect. 2.1, Fig. 0; differential rotation
// Sect. 3.4), replicate-padded spectrum rows, and the quiet velocity kernels.
//
// On a log-uniform grid a Doppler factor D = sqrt((1+beta)/(1-beta)) moves every pixel by the
// same amount s = ln D / Delta = atanh(beta) / Delta.  With j = ceil(s), the Eq. 11
// interpolation of output pixel m uses source pixels m-j and m-j+1 with the weight
//     w = (lambda_m - lambda'_{m-j}) / (lambda'_{m-j+1} - lambda'_{m-j})
//       = expm1((j - s) Delta) / expm1(Delta),
// independent of m.  A cell is therefore a two-tap kernel I(1-w) at offset j and I w at
// offset j-1, and cells with the same mu bin add up into one per-bin velocity kernel
// (the Toeplitz form of the disk sum).
//
// Integer decisions (visibility, mu bin) are computed with explicitly rounded FP64
// operations (no contraction) so they are reproducible bit for bit.
#include <cmath>

#include "soap_internal.cuh"

namespace soap {

struct MuTable {
    double v[SOAP_MAX_MU];
};

// atanh(x) = x + x^3/3 + x^5/5 + x^7/7 + ...; for |x| <= 1e-3 the omitted terms are below
// 1e-24 of x (GB300 FP64 is slow: four FMAs instead of a general atanh).
__device__ __forceinline__ double atanh_small(double x) {
    const double x2 = x * x;
    return fma(x * x2, fma(x2, fma(x2, 1.0 / 7.0, 1.0 / 5.0), 1.0 / 3.0), x);
}

// expm1(e) = e + e^2/2 + e^3/6 + ...; for |e| <= 1e-3 terms beyond e^6 are below 1e-21 of e.
__device__ __forceinline__ double expm1_small(double e) {
    return fma(e * e, fma(e, fma(e, fma(e, fma(e, 1.0 / 720.0, 1.0 / 120.0), 1.0 / 24.0), 1.0 / 6.0), 0.5), e);
}

// Nearest tabulated mu, ties to the lower index, as the first minimum of |mu - mu_b| in FP64.
// For a strictly increasing table the minimum lies next to the insertion point, so only a
// window around it is scanned (same answer as the full scan).
__device__ __forceinline__ int nearest_mu(double mu, int n_mu, const MuTable& mus, int sorted) {
    int b0 = 0, b1 = n_mu - 1;
    if (sorted) {
        int lo = 0, hi = n_mu;                  // first index with mu_b >= mu
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (mus.v[mid] < mu) lo = mid + 1; else hi = mid;
        }
        b0 = max(0, lo - 2);
        b1 = min(n_mu - 1, lo + 1);
    }
    int best = b0;
    double bd = fabs(__dsub_rn(mu, mus.v[b0]));
    for (int b = b0 + 1; b <= b1; b++) {
        double d = fabs(__dsub_rn(mu, mus.v[b]));
        if (d < bd) { bd = d; best = b; }
    }
    return best;
}

__global__ void k_cell_geometry(int N, double vsini, double sin_i, double cos_i, double alpha,
                                double u1, double u2, double delta, double expm1_delta,
                                int n_mu, MuTable mus, int mu_sorted, int tap_min, int tap_max, double* cell_I,
                                double* cell_w, double* cell_mu, int32_t* cell_j,
                                int32_t* cell_bin, unsigned int* flags) {
    int64_t NN = (int64_t)N * N;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < NN;
         c += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(c % N), j = (int)(c / N);
        double x = (double)(2 * i + 1 - N) / (double)N;
        double y = (double)(2 * j + 1 - N) / (double)N;
        double r2 = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
        if (!(r2 < 1.0)) {
            cell_I[c] = 0.0; cell_w[c] = 0.0; cell_mu[c] = 0.0; cell_j[c] = 0; cell_bin[c] = -1;
            continue;
        }
        double mu = __dsqrt_rn(__dsub_rn(1.0, r2));
        const int best = nearest_mu(mu, n_mu, mus, mu_sorted);
        double area = (2.0 / (double)N) * (2.0 / (double)N);
        double om = 1.0 - mu;
        double I = area * (1.0 - u1 * om - u2 * om * om);          // quadratic limb darkening
        double slat = y * sin_i + mu * cos_i;                        // sin(latitude) of the cell
        double v = vsini * x * (1.0 + alpha * slat * slat);          // x > 0 recedes
        const double beta = v / kCKms;
        double ab = fabs(beta) <= 1e-3 ? atanh_small(beta) : atanh(beta);    // ln D
        double s = ab / delta;
        double jd = ceil(s);
        int jt = (int)jd;
        const double e = fma(jd, delta, -ab);                        // (j - s) Delta
        double w = (delta <= 1e-3 ? expm1_small(e) : expm1(e)) / expm1_delta;
        if (jt - 1 < tap_min || jt > tap_max) {
            atomicOr(flags, kFlagTapRange);
            jt = jt < tap_min + 1 ? tap_min + 1 : tap_max;
        }
        cell_I[c] = I; cell_w[c] = w; cell_mu[c] = mu; cell_j[c] = jt; cell_bin[c] = best;
    }
}

// Fixed-point conversion: contributions are accumulated as 64-bit integers so that sums
// are exact and independent of the order the GPU happens to add them in.
__device__ __forceinline__ unsigned long long to_fixed(double v, double scale) {
    return (unsigned long long)__double2ll_rn(v * scale);
}

// quiet velocity kernels K_b[k] = sum_{c in bin b} I_c [(1-w_c) d(k, j_c) + w_c d(k, j_c - 1)]
__global__ void k_quiet_hist(int64_t NN, const double* cell_I, const double* cell_w,
                             const int32_t* cell_j, const int32_t* cell_bin, int tap_min,
                             int n_taps, int n_mu, double scale, long long* kout) {
    extern __shared__ long long hist[];
    int nb = n_mu * n_taps;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < NN;
         c += (int64_t)gridDim.x * blockDim.x) {
        int b = cell_bin[c];
        if (b < 0) continue;
        double I = cell_I[c], w = cell_w[c];
        int kk = cell_j[c] - tap_min;
        atomicAdd((unsigned long long*)&hist[b * n_taps + kk], to_fixed(I * (1.0 - w), scale));
        atomicAdd((unsigned long long*)&hist[b * n_taps + kk - 1], to_fixed(I * w, scale));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        if (hist[t]) atomicAdd((unsigned long long*)&kout[t], (unsigned long long)hist[t]);
}

__global__ void k_sum_intensity(int64_t NN, const double* cell_I, const int32_t* cell_bin,
                                double scale, long long* out2) {
    unsigned long long acc = 0, cnt = 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < NN;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (cell_bin[c] < 0) continue;
        acc += to_fixed(cell_I[c], scale);
        cnt += 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_down_sync(0xffffffffu, acc, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd((unsigned long long*)&out2[0], acc);
        atomicAdd((unsigned long long*)&out2[1], cnt);
    }
}

// Replicate-padded rows: dst[r][pad + n] = src[r][n]; left pad = src[r][0]; right pad =
// src[r][n_px-1].  Reading dst at pad + m - k for any tap k reproduces the clamped index
// min(max(m - k, 0), n_px - 1) of the interpolation's edge rule.
__global__ void k_pad_rows(const double* __restrict__ src, int64_t n_px, int64_t pad, int64_t row_len,
                           double* __restrict__ dst64, float* __restrict__ dst32) {
    const int64_t r = blockIdx.y;
    const double* s = src + r * n_px;
    double* d64 = dst64 + r * row_len;
    float* d32 = dst32 + r * row_len;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < row_len;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t n = e - pad;
        n = n < 0 ? 0 : (n >= n_px ? n_px - 1 : n);
        double v = __ldg(s + n);
        d64[e] = v;
        d32[e] = (float)v;
    }
}

static int grid_for(int64_t n, int threads, int cap = 152 * 16) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

soap_status pad_rows(soap_ctx* c, const double* src, double* dst64, float* dst32, int rows) {
    dim3 grid((unsigned)grid_for(c->row_len, 256, 64), (unsigned)rows);
    SOAP_TIMED(c, SOAP_TIMER_PAD_ROWS,
               k_pad_rows<<<grid, 256, 0, c->stream>>>(src, c->n_px, c->pad, c->row_len, dst64, dst32);
               SOAP_LAUNCHED(c));
    return SOAP_OK;
}

soap_status geometry_init(soap_ctx* c) {
    MuTable mus{};
    for (int b = 0; b < c->n_mu; b++) mus.v[b] = c->mu_values[b];
    double incl = c->incl_deg * (kPi / 180.0);
    int64_t NN = (int64_t)c->N * c->N;
    int tap_max = c->tap_min + c->n_taps - 1;
    cudaEvent_t tb = c->profiling ? timer_begin(c) : nullptr;
    k_cell_geometry<<<grid_for(NN, 256), 256, 0, c->stream>>>(
        c->N, c->vsini, std::sin(incl), std::cos(incl), c->alpha, c->u1, c->u2, c->delta,
        std::expm1(c->delta), c->n_mu, mus, c->mu_sorted, c->tap_min, tap_max, c->cell_I, c->cell_w, c->cell_mu,
        c->cell_j, c->cell_bin, c->flags);
    SOAP_LAUNCHED(c);
    // quiet kernels (exact integer sums)
    size_t nb = (size_t)c->n_mu * c->n_taps;
    SOAP_CUDA(cudaMemsetAsync(c->kq_fixed, 0, nb * sizeof(long long), c->stream));
    size_t smem = nb * sizeof(long long);
    if (smem > 48 * 1024)
        SOAP_CUDA(cudaFuncSetAttribute(k_quiet_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    double scale = std::ldexp(1.0, c->fx_bits);
    int g = grid_for(NN, 256, 152 * 2);
    k_quiet_hist<<<g, 256, smem, c->stream>>>(NN, c->cell_I, c->cell_w, c->cell_j, c->cell_bin,
                                              c->tap_min, c->n_taps, c->n_mu, scale, c->kq_fixed);
    SOAP_LAUNCHED(c);
    // visible-cell count and total intensity (read by soap_get_star_info)
    long long* d2 = c->sum_I_fixed;
    SOAP_CUDA(cudaMemsetAsync(d2, 0, 2 * sizeof(long long), c->stream));
    k_sum_intensity<<<grid_for(NN, 256, 152 * 4), 256, 0, c->stream>>>(NN, c->cell_I, c->cell_bin, scale, d2);
    SOAP_LAUNCHED(c);
    if (c->profiling) timer_end(c, SOAP_TIMER_GEOMETRY, tb);
    return SOAP_OK;
}

}  // namespace soap
