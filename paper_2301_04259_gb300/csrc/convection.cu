// convection.cu -- bisector injection (Sect. 4.3, the paper's Convec.model): the line bisector
// of each normalised local spectrum is replaced by a target one (per mu), shifting every point
// by the velocity of its normalised depth.
//
// A point n of depth d = clip(1 - F_n, 0, 1) moves by v = B_row(d) - B_orig(d) (km/s; the
// bisectors are tables over equally spaced depths, linear in between), i.e. to the pixel
// position u_n = n + atanh(v / c) / Delta of the log grid.  The moved points are re-sampled at
// the pixel centres linearly in wavelength, as in Eq. 11: for u_n <= m < u_n+1 the weight is
// expm1((m - u_n) Delta) / expm1((u_n+1 - u_n) Delta); outside the moved range the end values
// repeat.  The moved positions must stay increasing (flagged otherwise).
//
// Linear interpolation is linear, so the two tables merge on the host into one table of
// beta = (B_row - B_orig) / c per row (equal to the two-table form up to rounding), and the
// kernel looks up one value per point.
// k_bisectors: block = (tile of THREADS output pixels, row); the moved positions of the tile and
// a halo covering the largest shift are computed once into shared memory (points off the grid
// hold -inf / +inf), then each thread walks from its own pixel to its bracket: |u_n - n| is below
// halo - 1, so the walk takes about |shift| + 1 steps and never leaves the staged span.  FP64 (the
// local spectra are float64; |v|/c <= 1e-3 keeps atanh and expm1 in their short series).
#include <cmath>
#include <vector>

#include <math_constants.h>

#include "soap_internal.cuh"

namespace soap {

constexpr int kBisThreads = 256;
constexpr int kBisMaxHalo = 64;

__device__ __forceinline__ double table_at(const double* __restrict__ tab, int n_d, double d) {
    const double x = d * (double)(n_d - 1);
    int i = (int)x;                                     // d in [0, 1]: x >= 0
    if (i > n_d - 2) i = n_d - 2;
    const double f = x - (double)i;
    return fma(f, tab[i + 1] - tab[i], tab[i]);
}

// expm1(e) by its series up to e^K (K = 4: |e| <= 1e-4, truncation below 1e-18 of e; K = 6:
// |e| <= 1e-3, below 1e-20 of e), else the library function.
template <int K>
__device__ __forceinline__ double expm1_k(double e) {
    if constexpr (K == 4) {
        return fma(e * e, fma(e, fma(e, 1.0 / 24.0, 1.0 / 6.0), 0.5), e);
    } else if constexpr (K == 6) {
        return expm1_small(e);
    } else {
        return expm1(e);
    }
}

template <int K>
__global__ void __launch_bounds__(kBisThreads)
k_bisectors(const double* __restrict__ in, double* __restrict__ out, int n_px, int n_d,
            const double* __restrict__ beta_tab, double inv_delta, double delta, int halo, unsigned int* flags) {
    __shared__ double su[kBisThreads + 2 * kBisMaxHalo + 2];
    __shared__ double sf[kBisThreads + 2 * kBisMaxHalo + 2];
    const int r = blockIdx.y;
    const double* F = in + (int64_t)r * n_px;
    const double* T = beta_tab + (int64_t)r * n_d;
    const int m0 = blockIdx.x * kBisThreads;
    const int span = kBisThreads + 2 * halo + 1;          // points m0 - halo .. m0 + THREADS + halo
    for (int x = threadIdx.x; x < span; x += kBisThreads) {
        const int n = m0 - halo + x;
        double u = n < 0 ? -CUDART_INF : CUDART_INF, f = 0.0;
        if (n >= 0 && n < n_px) {
            f = F[n];
            const double d = fmin(fmax(1.0 - f, 0.0), 1.0);
            u = (double)n + atanh_small(table_at(T, n_d, d)) * inv_delta;
        }
        su[x] = u;
        sf[x] = f;
    }
    __syncthreads();
    // moved positions must increase (each pair checked once, by the block that owns its left point)
    for (int x = halo + threadIdx.x; x < halo + kBisThreads; x += kBisThreads) {
        const int n = m0 - halo + x;
        if (n >= 0 && n + 1 < n_px && !(su[x + 1] > su[x])) atomicOr(flags, kFlagOrder);
    }
    const int m = m0 + threadIdx.x;
    if (m >= n_px) return;
    // bracket: the largest point k with u_k <= m (-inf at n < 0 ends the walk down by n = m - halo + 1,
    // +inf at n >= n_px ends the walk up by n = m + halo - 1)
    const double mm = (double)m;
    int k = threadIdx.x + halo;
    while (su[k] > mm) k--;
    while (su[k + 1] <= mm) k++;
    double val;
    const int nk = m0 - halo + k;
    if (nk < 0) {
        val = F[0];                                       // before the first moved point
    } else if (nk >= n_px - 1) {
        val = F[n_px - 1];                                // at or past the last moved point
    } else {
        const double w = expm1_k<K>((mm - su[k]) * delta) / expm1_k<K>((su[k + 1] - su[k]) * delta);
        val = fma(w, sf[k + 1] - sf[k], sf[k]);
    }
    out[(int64_t)r * n_px + m] = val;
}

soap_status inject_bisectors(soap_ctx* c, const double* in, double* out, int n_rows, const double* bis_host,
                             const double* orig_host, int n_d) {
    if (n_rows <= 0) return SOAP_OK;
    double vmax = 0.0;
    for (int64_t i = 0; i < (int64_t)n_rows * n_d; i++) {
        if (!std::isfinite(bis_host[i])) { set_error("bisector table entry %lld not finite", (long long)i); return SOAP_EINVAL; }
        vmax = std::max(vmax, std::fabs(bis_host[i]));
    }
    double omax = 0.0;
    for (int i = 0; i < n_d; i++) {
        if (!std::isfinite(orig_host[i])) { set_error("original bisector entry %d not finite", i); return SOAP_EINVAL; }
        omax = std::max(omax, std::fabs(orig_host[i]));
    }
    const double vbound = vmax + omax;                    // km/s
    if (!(vbound / kCKms <= 1e-3)) { set_error("bisector velocities above 1e-3 c"); return SOAP_ERANGE; }
    const double shift = std::atanh(vbound / kCKms) / c->delta;
    const int halo = (int)std::ceil(shift) + 2;
    if (halo > kBisMaxHalo) {
        set_error("bisector shifts of %.1f pixels exceed %d", shift, kBisMaxHalo - 2);
        return SOAP_ERANGE;
    }
    std::vector<double> beta((size_t)n_rows * n_d);
    for (int r = 0; r < n_rows; r++)
        for (int j = 0; j < n_d; j++)
            beta[(size_t)r * n_d + j] = (bis_host[(size_t)r * n_d + j] - orig_host[j]) / kCKms;
    SOAP_TRY(ensure(c->bis_tab, beta.size() * sizeof(double)));
    SOAP_TRY(upload_small(c, c->bis_tab.p, beta.data(), beta.size() * sizeof(double)));
    // largest expm1 argument: (u_n+1 - u_n) Delta <= (1 + 2 shift) Delta
    const double emax = (1.0 + 2.0 * shift) * c->delta;
    dim3 grid((unsigned)((c->n_px + kBisThreads - 1) / kBisThreads), (unsigned)n_rows);
    auto launch = [&](auto kern) {
        SOAP_TIMED(c, SOAP_TIMER_BISECTORS,
                   (kern<<<grid, kBisThreads, 0, c->stream>>>(in, out, (int)c->n_px, n_d, c->bis_tab.as<double>(),
                                                              1.0 / c->delta, c->delta, halo, c->flags)));
    };
    if (emax <= 1e-4) launch(k_bisectors<4>);
    else if (emax <= 1e-3) launch(k_bisectors<6>);
    else launch(k_bisectors<0>);
    SOAP_CUDA(cudaGetLastError());
    SOAP_LAUNCHED(c);
    return SOAP_OK;
}

}  // namespace soap
