// instrument.cu -- instrumental resolution (Sect. 3.3, after Eq. 4; Alg. 5): each integrated
// spectrum is degraded to the instrument's resolving power R.
//
// The paper does not give the method.  Line-spread function: a Gaussian of FWHM lambda / R.  On
// the log-uniform grid that is a fixed width in pixels, FWHM = 1 / (R Delta), and the discrete
// kernel has one tap per pixel, the Gaussian's mass over that pixel, for |k| <= K =
// ceil(6 sigma) + 1, renormalised to unit sum:
//     out[m] = sum_k g[k] F[clamp(m - k)],
// source indices clamped to the grid (the end values repeat, as for the Doppler shifts).  The
// taps are computed once on the host in FP64.
//
// k_lsf_win: a block owns a tile of THREADS x E consecutive pixels of one spectrum, staged with
// its 2K halo in shared memory; a thread owns E consecutive outputs and keeps the E + 2K inputs
// they need in registers (16-byte shared loads), so each staged value is read from shared memory
// about once.  HBM traffic: each spectrum read once and written once.
#include <cmath>
#include <vector>

#include "soap_internal.cuh"

namespace soap {

soap_status lsf_taps(double resolving_power, double delta, std::vector<double>& g, int& K) {
    if (!(resolving_power > 0) || !std::isfinite(resolving_power)) {
        set_error("resolving power must be finite and > 0");
        return SOAP_EINVAL;
    }
    const double sigma = 1.0 / (resolving_power * delta * 2.0 * std::sqrt(2.0 * std::log(2.0)));
    if (!(sigma <= 800.0)) {                                  // K <= 4802: the generic kernel's tile fits
        set_error("resolving power %g gives a line-spread function of sigma > 800 pixels", resolving_power);
        return SOAP_ERANGE;
    }
    K = (int)std::ceil(6.0 * sigma) + 1;
    const double s2 = sigma * std::sqrt(2.0);
    std::vector<double> half((size_t)K + 1);
    half[0] = std::erf(0.5 / s2);
    for (int k = 1; k <= K; k++) half[(size_t)k] = 0.5 * (std::erfc((k - 0.5) / s2) - std::erfc((k + 0.5) / s2));
    g.assign(2 * (size_t)K + 1, 0.0);
    for (int k = -K; k <= K; k++) g[(size_t)(k + K)] = half[(size_t)std::abs(k)];
    double tot = 0.0;
    for (double v : g) tot += v;
    for (double& v : g) v /= tot;
    return SOAP_OK;
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using V = float4;
    static constexpr int n = 4;
    __device__ static void get(const V& v, float* d) { d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w; }
    __device__ static V make(const float* a) { return make_float4(a[0], a[1], a[2], a[3]); }
};
template <>
struct Vec16<double> {
    using V = double2;
    static constexpr int n = 2;
    __device__ static void get(const V& v, double* d) { d[0] = v.x; d[1] = v.y; }
    __device__ static V make(const double* a) { return make_double2(a[0], a[1]); }
};

// Windowed form for K <= KMAX.  Shared: the tile [m0 - K, m0 + THREADS E + K) (clamped source
// indices), padded to whole 16-byte vectors, and the 2K + 1 taps.
template <typename T, int E, int KMAX, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_lsf_win(const T* __restrict__ in, T* __restrict__ out, int64_t n_px, int K, const T* __restrict__ taps) {
    constexpr int VN = Vec16<T>::n;
    constexpr int WIN = E + 2 * KMAX;                       // register window (upper bound)
    constexpr int NV = (WIN + VN - 1) / VN;
    extern __shared__ __align__(16) unsigned char lsf_raw[];
    T* s = reinterpret_cast<T*>(lsf_raw);
    const int TP = THREADS * E;
    const int span = TP + 2 * K;
    const int span_pad = (TP + 2 * KMAX + VN - 1) / VN * VN + VN;
    T* g = s + span_pad;
    const T* src = in + (int64_t)blockIdx.y * n_px;
    T* dst = out + (int64_t)blockIdx.y * n_px;
    const int64_t m0 = (int64_t)blockIdx.x * TP;
    // K is a multiple of VN here (taps padded with zeros), so an interior tile starts on a
    // 16-byte boundary when the row does: then it is staged with 16-byte loads
    const bool interior = m0 - K >= 0 && m0 - K + span <= n_px &&
                          (reinterpret_cast<uintptr_t>(src + (m0 - K)) & 15) == 0;
    if (interior) {
        using V = typename Vec16<T>::V;
        const V* sv_src = reinterpret_cast<const V*>(src + (m0 - K));
        V* sv_dst = reinterpret_cast<V*>(s);
        const int nv = span / VN;                          // span = TP + 2K is a multiple of VN
        for (int x = threadIdx.x; x < nv; x += THREADS) sv_dst[x] = __ldg(sv_src + x);
        for (int x = span + threadIdx.x; x < span_pad; x += THREADS) s[x] = T(0);
    } else {
        for (int x = threadIdx.x; x < span_pad; x += THREADS) {
            T v = T(0);
            if (x < span) {
                int64_t n = m0 - K + x;
                n = n < 0 ? 0 : (n >= n_px ? n_px - 1 : n);
                v = __ldg(src + n);
            }
            s[x] = v;
        }
    }
    for (int k = threadIdx.x; k <= 2 * K; k += THREADS) g[k] = taps[k];
    __syncthreads();
    // window w[j] = s[E t + j], j < E + 2K (16-byte loads; E t is a multiple of VN)
    T w[NV * VN];
    const typename Vec16<T>::V* sv = reinterpret_cast<const typename Vec16<T>::V*>(s + E * threadIdx.x);
#pragma unroll
    for (int q = 0; q < NV; q++) Vec16<T>::get(sv[q], w + q * VN);
    T acc[E];
#pragma unroll
    for (int i = 0; i < E; i++) acc[i] = T(0);
    // out[m0 + E t + i] = sum_{k=-K..K} g[K + k] s[E t + i + K - k] = sum_j g[2K - j] w[i + j]
    // (j unrolled to 2 KMAX so that w is indexed by constants; the taps past 2K are skipped)
#pragma unroll
    for (int j = 0; j <= 2 * KMAX; j++) {
        if (j > 2 * K) break;
        const T gj = g[2 * K - j];
#pragma unroll
        for (int i = 0; i < E; i++) acc[i] = fma(gj, w[i + j], acc[i]);
    }
    const int64_t mt = m0 + E * threadIdx.x;
    if (mt + E <= n_px && (reinterpret_cast<uintptr_t>(dst + mt) & 15) == 0) {   // whole 16-byte vectors
        typename Vec16<T>::V* d = reinterpret_cast<typename Vec16<T>::V*>(dst + mt);
#pragma unroll
        for (int q = 0; q < E / VN; q++) d[q] = Vec16<T>::make(acc + q * VN);
    } else {
#pragma unroll
        for (int i = 0; i < E; i++)
            if (mt + i < n_px) dst[mt + i] = acc[i];
    }
}

// Generic form (any K): a thread owns pixels m0 + t + i THREADS and reads every tap's source
// from the staged tile (consecutive threads, consecutive addresses).
template <typename T, int E, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_lsf_gen(const T* __restrict__ in, T* __restrict__ out, int64_t n_px, int K, const T* __restrict__ taps) {
    extern __shared__ __align__(16) unsigned char lsf_raw[];
    T* s = reinterpret_cast<T*>(lsf_raw);
    const int TP = THREADS * E;
    const int span = TP + 2 * K;
    T* g = s + span;
    const T* src = in + (int64_t)blockIdx.y * n_px;
    T* dst = out + (int64_t)blockIdx.y * n_px;
    const int64_t m0 = (int64_t)blockIdx.x * TP;
    for (int x = threadIdx.x; x < span; x += THREADS) {
        int64_t n = m0 - K + x;
        n = n < 0 ? 0 : (n >= n_px ? n_px - 1 : n);
        s[x] = __ldg(src + n);
    }
    for (int k = threadIdx.x; k <= 2 * K; k += THREADS) g[k] = taps[k];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < E; i++) {
        const int x = threadIdx.x + i * THREADS;
        T acc = T(0);
        for (int j = 0; j <= 2 * K; j++) acc = fma(g[2 * K - j], s[x + j], acc);
        const int64_t m = m0 + x;
        if (m < n_px) dst[m] = acc;
    }
}

#ifndef SOAP_LSF_E
#define SOAP_LSF_E 8
#endif
constexpr int kLsfE = SOAP_LSF_E, kLsfKmax = 12, kLsfThreads = 128;

template <typename T>
static soap_status launch_lsf_t(soap_ctx* c, const T* in, T* out, int64_t n_spec) {
    const int K = c->lsf_K;
    constexpr int VN = 16 / (int)sizeof(T);
    const bool win = (K + VN - 1) / VN * VN <= kLsfKmax;
    // windowed form: the taps padded with zeros to round_up(K, VN) each side (the extra terms add
    // exact zeros), so that tiles start on 16-byte boundaries
    const int Kw = win ? (K + VN - 1) / VN * VN : K;
    const size_t off = win ? (sizeof(T) == 8 ? c->lsf_offp64 : c->lsf_offp32) : (sizeof(T) == 8 ? 0 : c->lsf_off32);
    const T* taps = reinterpret_cast<const T*>(c->lsf_taps.as<char>() + off);
    const int TP = kLsfThreads * kLsfE;
    const int64_t tiles = (c->n_px + TP - 1) / TP;
    for (int64_t s0 = 0; s0 < n_spec; s0 += 65535) {
        const unsigned ny = (unsigned)std::min<int64_t>(65535, n_spec - s0);
        dim3 grid((unsigned)tiles, ny);
        const T* i0 = in + s0 * c->n_px;
        T* o0 = out + s0 * c->n_px;
        if (win) {
            const int span_pad = (TP + 2 * kLsfKmax + VN - 1) / VN * VN + VN;
            const size_t smem = ((size_t)span_pad + 2 * kLsfKmax + 1) * sizeof(T);
            SOAP_TIMED(c, SOAP_TIMER_LSF,
                       k_lsf_win<T, kLsfE, kLsfKmax, kLsfThreads><<<grid, kLsfThreads, smem, c->stream>>>(
                           i0, o0, c->n_px, Kw, taps);
                       SOAP_LAUNCHED(c));
        } else {
            const size_t smem = ((size_t)TP + 4 * K + 1) * sizeof(T);
            if (smem > 48 * 1024)
                SOAP_CUDA(cudaFuncSetAttribute(k_lsf_gen<T, kLsfE, kLsfThreads>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            SOAP_TIMED(c, SOAP_TIMER_LSF,
                       k_lsf_gen<T, kLsfE, kLsfThreads><<<grid, kLsfThreads, smem, c->stream>>>(
                           i0, o0, c->n_px, K, taps);
                       SOAP_LAUNCHED(c));
        }
    }
    return SOAP_OK;
}

soap_status launch_lsf(soap_ctx* c, const void* in, void* out, int f32, int64_t n_spec) {
    if (n_spec <= 0) return SOAP_OK;
    if (f32) return launch_lsf_t<float>(c, static_cast<const float*>(in), static_cast<float*>(out), n_spec);
    return launch_lsf_t<double>(c, static_cast<const double*>(in), static_cast<double*>(out), n_spec);
}

soap_status set_instrument(soap_ctx* c, double resolving_power) {
    if (resolving_power == 0.0) {
        c->lsf_K = -1;
        c->lsf_R = 0.0;
        return SOAP_OK;
    }
    std::vector<double> g;
    int K = 0;
    SOAP_TRY(lsf_taps(resolving_power, c->delta, g, K));
    if (K >= c->n_px) {
        set_error("the line-spread function (%d taps each side) is wider than the grid", K);
        return SOAP_ERANGE;
    }
    const size_t n = g.size();
    // zero-padded copies for the windowed form: K rounded up to 2 (float64) and 4 (float32)
    auto padded = [&](int Kp) {
        std::vector<double> gp(2 * (size_t)Kp + 1, 0.0);
        for (int k = -K; k <= K; k++) gp[(size_t)(k + Kp)] = g[(size_t)(k + K)];
        return gp;
    };
    const std::vector<double> gp64 = padded((K + 1) / 2 * 2), gp32d = padded((K + 3) / 4 * 4);
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t off32 = al(n * sizeof(double));
    const size_t offp64 = al(off32 + n * sizeof(float));
    const size_t offp32 = al(offp64 + gp64.size() * sizeof(double));
    SOAP_TRY(ensure(c->lsf_taps, offp32 + gp32d.size() * sizeof(float)));
    std::vector<float> g32(n), gp32(gp32d.size());
    for (size_t i = 0; i < n; i++) g32[i] = (float)g[i];
    for (size_t i = 0; i < gp32d.size(); i++) gp32[i] = (float)gp32d[i];
    char* base = c->lsf_taps.as<char>();
    SOAP_TRY(upload_small(c, base, g.data(), n * sizeof(double)));
    SOAP_TRY(upload_small(c, base + off32, g32.data(), n * sizeof(float)));
    SOAP_TRY(upload_small(c, base + offp64, gp64.data(), gp64.size() * sizeof(double)));
    SOAP_TRY(upload_small(c, base + offp32, gp32.data(), gp32.size() * sizeof(float)));
    c->lsf_off32 = off32;
    c->lsf_offp64 = offp64;
    c->lsf_offp32 = offp32;
    c->lsf_K = K;
    c->lsf_R = resolving_power;
    return SOAP_OK;
}

}  // namespace soap
