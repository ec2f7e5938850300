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
    float mid[SOAP_MAX_MU];   // (mu_b + mu_b+1) / 2 rounded to float (used when fast32 is set)
    int fast32;               // strictly increasing, neighbours at least 1e-4 apart
};

// Nearest tabulated mu, ties to the lower index, as the first minimum of |mu - mu_b| in FP64.
// For a strictly increasing table the minimum lies next to the insertion point, so only a
// window around it is scanned (same answer as the full scan).  With fast32 the bin is first
// read off the FP32 midpoints: mu and the midpoints are within 6e-8 of their float roundings,
// so a float mu farther than 1e-6 from both midpoints around it lies on the same sides of the
// exact midpoints, where the FP64 comparison decides the same bin (the FP64 pipe is the
// geometry kernel's limit, the FP32 compares cost nothing); closer ones take the FP64 path.
__device__ __forceinline__ int nearest_mu(double mu, int n_mu, const MuTable& mus, int sorted) {
    if (mus.fast32) {
        const float mf = __double2float_rn(mu);
        int lo = 0, hi = n_mu - 1;              // number of midpoints below mf
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (mus.mid[mid] < mf) lo = mid + 1; else hi = mid;
        }
        const bool near = (lo > 0 && fabsf(mf - mus.mid[lo - 1]) < 1e-6f) ||
                          (lo < n_mu - 1 && fabsf(mf - mus.mid[lo]) < 1e-6f);
        if (!near) return lo;
    }
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

// hist[key] += v for every lane with on set.  Lanes of a warp with equal keys in consecutive
// lanes (neighbouring cells of a row mostly share their mu bin and velocity offset) are summed
// first by a segmented scan, and the last lane of each run adds the run's sum: one shared-memory
// atomic per run instead of one per cell.  The sums are integers, so the result is exact in any
// order.  Every lane of the warp must call it.
__device__ __forceinline__ void hist_add_runs(long long* hist, int key, unsigned long long v, bool on) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int k = on ? key : -1;
    const int kprev = __shfl_up_sync(full, k, 1);
    const int knext = __shfl_down_sync(full, k, 1);
    int start = (lane == 0 || kprev != k) ? lane : 0;          // first lane of this lane's run
    for (int o = 1; o < 32; o <<= 1) start = max(start, __shfl_up_sync(full, start, o));
    unsigned long long sum = on ? v : 0ull;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(full, sum, o);
        if (lane - o >= start) sum += t;
    }
    if (on && (lane == 31 || knext != k)) atomicAdd((unsigned long long*)&hist[k], sum);
}

// One block per (row j, 128 columns).  Besides the geometry it stores, per cell, the two
// fixed-point contributions fx(I (1-w)) and fx(I w) of its two-tap kernel (reused by every
// phase), an FP32 copy of mu (for the FP32 membership pre-test), and adds the cell to the quiet
// velocity kernels (shared-memory 64-bit integer sums, then one atomic per non-zero bin) and
// to the total intensity.  Integer sums are exact, so the result does not depend on order.
// SERIES: every |beta| and the grid step are at most 1e-3 (decided on the host), so atanh and
// expm1 are their short series; otherwise the library functions (only one form is compiled into
// each instance, so no cell evaluates both).
template <bool SERIES>
__global__ void __launch_bounds__(128)
k_geometry(int N, double vsini, double sin_i, double cos_i, double alpha, double u1, double u2,
           double inv_c, double inv_delta, double delta, double inv_expm1_delta, int n_mu,
           MuTable mus, int mu_sorted, int tap_min, int tap_max, int n_taps, double scale,
           double* cell_I, double* cell_w, double* cell_mu, float* cell_mu32, int32_t* cell_j,
           int32_t* cell_bin, long long* cell_k0, long long* cell_k1, long long* kq_fixed,
           long long* sum2, long long* qtoff, int* qgstart, double* qc64, float* qc32, int q_max_taps,
           int64_t row_len, int64_t pad, int fx_bits, int* counter, unsigned int* flags,
           const double* __restrict__ cell_x, double area, TapGroup* qgrp, int* qgrp_start) {
    extern __shared__ long long hist[];                  // [n_mu][n_taps]
    const int nb = n_mu * n_taps;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) hist[t] = 0;
    const int j = blockIdx.y;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long sumI = 0, cnt = 0;
    int hkey = 0;                                      // the cell's (bin, tap) entry and its two taps
    unsigned long long hk0 = 0, hk1 = 0;
    bool hon = false;
    if (i < N) {
        const int64_t c = (int64_t)j * N + i;
        const double x = cell_x[i];                                        // (2 i + 1 - N) / N
        const double y = cell_x[j];
        const double r2 = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
        if (!(r2 < 1.0)) {
            cell_I[c] = 0.0; cell_w[c] = 0.0; cell_mu[c] = 0.0; cell_mu32[c] = 0.0f;
            cell_j[c] = 0; cell_bin[c] = -1; cell_k0[c] = 0; cell_k1[c] = 0;
        } else {
            const double mu = __dsqrt_rn(__dsub_rn(1.0, r2));
            const int best = nearest_mu(mu, n_mu, mus, mu_sorted);
            const double om = 1.0 - mu;
            const double I = area * (1.0 - u1 * om - u2 * om * om);      // quadratic limb darkening
            const double slat = y * sin_i + mu * cos_i;                    // sin(latitude) of the cell
            // x > 0 recedes; rigid rotation (alpha = 0) skips the latitude term, 1 + 0 s^2 = 1 exactly
            const double v = alpha != 0.0 ? vsini * x * (1.0 + alpha * slat * slat) : vsini * x;
            const double beta = v * inv_c;
            const double ab = SERIES ? atanh_small(beta) : atanh(beta);    // ln D
            const double jd = ceil(ab * inv_delta);                        // j = ceil(s), s = ln D / Delta
            int jt = (int)jd;
            const double e = fma(jd, delta, -ab);                          // (j - s) Delta
            const double w = (SERIES ? expm1_small(e) : expm1(e)) * inv_expm1_delta;
            if (jt - 1 < tap_min || jt > tap_max) {
                atomicOr(flags, kFlagTapRange);
                jt = jt < tap_min + 1 ? tap_min + 1 : tap_max;
            }
            const long long k0 = __double2ll_rn(I * (1.0 - w) * scale);
            const long long k1 = __double2ll_rn(I * w * scale);
            cell_I[c] = I; cell_w[c] = w; cell_mu[c] = mu; cell_mu32[c] = (float)mu;
            cell_j[c] = jt; cell_bin[c] = best; cell_k0[c] = k0; cell_k1[c] = k1;
            hkey = best * n_taps + (jt - tap_min);
            hk0 = (unsigned long long)k0;
            hk1 = (unsigned long long)k1;
            hon = true;
            sumI = (unsigned long long)__double2ll_rn(I * scale);
            cnt = 1;
        }
    }
    hist_add_runs(hist, hkey, hk0, hon);
    hist_add_runs(hist, hkey - 1, hk1, hon);
    for (int o = 16; o > 0; o >>= 1) {
        sumI += __shfl_down_sync(0xffffffffu, sumI, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0 && cnt) {
        atomicAdd((unsigned long long*)&sum2[0], sumI);
        atomicAdd((unsigned long long*)&sum2[1], cnt);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        if (hist[t]) atomicAdd((unsigned long long*)&kq_fixed[t], (unsigned long long)hist[t]);
    // the last block to finish builds the quiet tap table (one "phase", one group)
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int t = atomicAdd(counter, 1);
        s_last = t == (int)(gridDim.x * gridDim.y) - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        build_taps_dev(kq_fixed, 0, 1, 1, n_mu, n_taps, tap_min, 1, 0, 1.0 / scale, fx_bits, row_len, pad, qtoff,
                       qgstart, qc64, qc32, q_max_taps, hist, flags, nullptr, qgrp, qgrp_start);
    }
}

// Replicate-padded rows: dst[r][pad + n] = src[r][n]; left pad = src[r][0]; right pad =
// src[r][n_px-1].  Reading dst at pad + m - k for any tap k reproduces the clamped index
// min(max(m - k, 0), n_px - 1) of the interpolation's edge rule.
// Warp-cooperative: one warp covers 32 x kPadE consecutive outputs of a row, lane l taking
// elements l, l + 32, ..., so every load and store instruction covers contiguous bytes (the
// source is shifted by pad against the destination, so per-thread vectors would not align).
// Indices within a row are 32-bit (row_len < 2^31).
constexpr int kPadE = 8;

__global__ void k_pad_rows(const double* __restrict__ src, int n_px, int pad, int row_len,
                           double* __restrict__ dst64, float* __restrict__ dst32) {
    const int64_t r = blockIdx.y;
    const double* s = src + r * n_px;
    double* d64 = dst64 + r * row_len;
    float* d32 = dst32 + r * row_len;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int stride = gridDim.x * wpb * 32 * kPadE;
    for (int base = (blockIdx.x * wpb + (threadIdx.x >> 5)) * 32 * kPadE; base < row_len; base += stride) {
        double v[kPadE];
#pragma unroll
        for (int t = 0; t < kPadE; t++) {
            const int n = min(max(base + 32 * t + lane - pad, 0), n_px - 1);
            v[t] = __ldg(s + n);
        }
#pragma unroll
        for (int t = 0; t < kPadE; t++) {
            const int e = base + 32 * t + lane;
            if (e < row_len) {
                d64[e] = v[t];
                d32[e] = (float)v[t];
            }
        }
    }
}

// float32 local spectra: the float32 rows only
__global__ void k_pad_rows32(const float* __restrict__ src, int n_px, int pad, int row_len,
                             float* __restrict__ dst32) {
    const int64_t r = blockIdx.y;
    const float* s = src + r * n_px;
    float* d32 = dst32 + r * row_len;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int stride = gridDim.x * wpb * 32 * kPadE;
    for (int base = (blockIdx.x * wpb + (threadIdx.x >> 5)) * 32 * kPadE; base < row_len; base += stride) {
        float v[kPadE];
#pragma unroll
        for (int t = 0; t < kPadE; t++) {
            const int n = min(max(base + 32 * t + lane - pad, 0), n_px - 1);
            v[t] = __ldg(s + n);
        }
#pragma unroll
        for (int t = 0; t < kPadE; t++) {
            const int e = base + 32 * t + lane;
            if (e < row_len) d32[e] = v[t];
        }
    }
}

// The same rows with 16-byte accesses, when pad and n_px are multiples of 4 and both arrays are
// 16-byte aligned: each element group e .. e+3 of a row is either inside the spectrum (one
// 16-byte load) or touches an end (the clamped indices, one by one).  Block (x, row): four
// groups per thread per iteration, loads first.
constexpr int kPadV = 4;

__global__ void k_pad_rows32v(const float* __restrict__ src, int n_px, int pad, int row_len,
                              float* __restrict__ dst32) {
    const int64_t r = blockIdx.y;
    const float* s = src + r * n_px;
    float4* d = reinterpret_cast<float4*>(dst32 + r * row_len);
    const int nq = row_len / 4;
    const int step = gridDim.x * blockDim.x;
    for (int q0 = blockIdx.x * blockDim.x + threadIdx.x; q0 < nq; q0 += kPadV * step) {
        float4 v[kPadV];
#pragma unroll
        for (int u = 0; u < kPadV; u++) {
            const int q = q0 + u * step;
            const int n = 4 * q - pad;
            if (q >= nq) {
                v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else if (n >= 0 && n + 3 < n_px) {
                v[u] = __ldg(reinterpret_cast<const float4*>(s + n));
            } else {
                v[u].x = __ldg(s + min(max(n, 0), n_px - 1));
                v[u].y = __ldg(s + min(max(n + 1, 0), n_px - 1));
                v[u].z = __ldg(s + min(max(n + 2, 0), n_px - 1));
                v[u].w = __ldg(s + min(max(n + 3, 0), n_px - 1));
            }
        }
#pragma unroll
        for (int u = 0; u < kPadV; u++) {
            const int q = q0 + u * step;
            if (q < nq) d[q] = v[u];
        }
    }
}

static int grid_for(int64_t n, int threads, int cap = 152 * 16) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

soap_status pad_rows(soap_ctx* c, const double* src, double* dst64, float* dst32, int rows) {
    dim3 grid((unsigned)grid_for(c->row_len / kPadE, 256, 64), (unsigned)rows);
    SOAP_TIMED(c, SOAP_TIMER_PAD_ROWS,
               k_pad_rows<<<grid, 256, 0, c->stream>>>(src, (int)c->n_px, (int)c->pad, (int)c->row_len,
                                                       dst64, dst32);
               SOAP_LAUNCHED(c));
    return SOAP_OK;
}

soap_status pad_rows32(soap_ctx* c, const float* src, float* dst32, int rows) {
    const bool vec = c->pad % 4 == 0 && c->n_px % 4 == 0 && c->row_len % 4 == 0 &&
                     ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst32)) & 15) == 0;
    if (vec) {
        // about 8 blocks of 256 threads per SM over all rows
        const int bx = std::max(1, std::min((int)((c->row_len / 4 + 255) / 256), (152 * 8 + rows - 1) / rows));
        dim3 vgrid((unsigned)bx, (unsigned)rows);
        SOAP_TIMED(c, SOAP_TIMER_PAD_ROWS,
                   k_pad_rows32v<<<vgrid, 256, 0, c->stream>>>(src, (int)c->n_px, (int)c->pad, (int)c->row_len,
                                                               dst32);
                   SOAP_LAUNCHED(c));
        return SOAP_OK;
    }
    dim3 grid((unsigned)grid_for(c->row_len / kPadE, 256, 64), (unsigned)rows);
    SOAP_TIMED(c, SOAP_TIMER_PAD_ROWS,
               k_pad_rows32<<<grid, 256, 0, c->stream>>>(src, (int)c->n_px, (int)c->pad, (int)c->row_len,
                                                         dst32);
               SOAP_LAUNCHED(c));
    return SOAP_OK;
}

// The geometry depends only on the star: it runs on the auxiliary stream after everything
// queued so far on the main stream (which may still read the previous geometry), so that the
// main stream's next kernels (padded rows, contrast, region boxes) overlap it.  Readers of the
// cell tables and quiet kernels call join_geometry first.
soap_status geometry_init(soap_ctx* c) {
    MuTable mus{};
    for (int b = 0; b < c->n_mu; b++) mus.v[b] = c->mu_values[b];
    mus.fast32 = c->mu_sorted;
    for (int b = 0; b + 1 < c->n_mu; b++) {
        mus.mid[b] = (float)(0.5 * (c->mu_values[b] + c->mu_values[b + 1]));
        if (!(c->mu_values[b + 1] - c->mu_values[b] >= 1e-4)) mus.fast32 = 0;
    }
    double incl = c->incl_deg * (kPi / 180.0);
    int tap_max = c->tap_min + c->n_taps - 1;
    size_t nb = (size_t)c->n_mu * c->n_taps;
    const double scale = std::ldexp(1.0, c->fx_bits);
    size_t smem = nb * sizeof(long long);
    // largest |beta| = vsini (1 + |alpha|) / c over the disk (|x| < 1, sin^2(latitude) <= 1)
    const bool series = c->vsini * (1.0 + std::fabs(c->alpha)) / kCKms <= 1e-3 && c->delta <= 1e-3;
    auto kern = series ? k_geometry<true> : k_geometry<false>;
    SOAP_TRY(fit_dynamic_smem(kern, smem));
    SOAP_CUDA(cudaEventRecord(c->ev_fork, c->stream));
    SOAP_CUDA(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    {
        OnStream on(c, c->aux);
        cudaEvent_t tb = c->profiling ? timer_begin(c) : nullptr;
        SOAP_CUDA(cudaMemsetAsync(c->kq_fixed, 0, nb * sizeof(long long), c->stream));
        SOAP_CUDA(cudaMemsetAsync(c->sum_I_fixed, 0, 2 * sizeof(long long), c->stream));
        SOAP_CUDA(cudaMemsetAsync(c->geo_counter, 0, sizeof(int), c->stream));
        dim3 grid((unsigned)((c->N + 127) / 128), (unsigned)c->N);
        kern<<<grid, 128, smem, c->stream>>>(
            c->N, c->vsini, std::sin(incl), std::cos(incl), c->alpha, c->u1, c->u2, 1.0 / kCKms,
            1.0 / c->delta, c->delta, 1.0 / std::expm1(c->delta), c->n_mu, mus, c->mu_sorted, c->tap_min,
            tap_max, c->n_taps, scale, c->cell_I, c->cell_w, c->cell_mu, c->cell_mu32, c->cell_j,
            c->cell_bin, c->cell_k0, c->cell_k1, c->kq_fixed, c->sum_I_fixed, c->qtoff, c->qgstart, c->qc64,
            c->qc32, c->n_mu * SOAP_MAX_TAPS, c->row_len, c->pad, c->fx_bits, c->geo_counter, c->flags,
            c->cell_x, (2.0 / (double)c->N) * (2.0 / (double)c->N), c->qgrp, c->qgrp_start);
        SOAP_LAUNCHED(c);
        if (c->profiling) timer_end(c, SOAP_TIMER_GEOMETRY, tb);
        SOAP_CUDA(cudaEventRecord(c->ev_geo, c->stream));
    }
    c->geo_pending = true;
    c->geo_version++;
    return SOAP_OK;
}

soap_status join_geometry(soap_ctx* c) {
    if (!c->geo_pending) return SOAP_OK;
    SOAP_CUDA(cudaStreamWaitEvent(c->stream, c->ev_geo, 0));
    c->geo_pending = false;
    return SOAP_OK;
}

}  // namespace soap
