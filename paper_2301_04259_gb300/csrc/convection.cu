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
// k_bisectors: block = (tile of THREADS output pixels, row); the moved positions of the tile and
// a halo covering the largest shift are computed once into shared memory, then each thread finds
// its bracket there.  FP64 (the local spectra are float64; |v|/c <= 1e-3 keeps atanh and expm1 in
// their short series).
#include <cmath>
#include <vector>

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

__global__ void __launch_bounds__(kBisThreads)
k_bisectors(const double* __restrict__ in, double* __restrict__ out, int n_px, int n_d,
            const double* __restrict__ bis, const double* __restrict__ orig, double inv_c,
            double inv_delta, double delta, int halo, unsigned int* flags) {
    __shared__ double su[kBisThreads + 2 * kBisMaxHalo + 2];
    __shared__ double sf[kBisThreads + 2 * kBisMaxHalo + 2];
    const int r = blockIdx.y;
    const double* F = in + (int64_t)r * n_px;
    const double* B = bis + (int64_t)r * n_d;
    const int m0 = blockIdx.x * kBisThreads;
    const int span = kBisThreads + 2 * halo + 1;          // points m0 - halo .. m0 + THREADS + halo
    for (int x = threadIdx.x; x < span; x += kBisThreads) {
        const int n = m0 - halo + x;
        double u = 0.0, f = 0.0;
        if (n >= 0 && n < n_px) {
            f = F[n];
            const double d = fmin(fmax(1.0 - f, 0.0), 1.0);
            const double v = table_at(B, n_d, d) - table_at(orig, n_d, d);
            u = (double)n + atanh_small(v * inv_c) * inv_delta;
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
    // largest point n in m - halo .. m + halo with u_n <= m: the bracket (|u_n - n| < halo - 1)
    const double mm = (double)m;
    int k = -1;
    for (int x = threadIdx.x; x <= threadIdx.x + 2 * halo; x++) {
        const int n = m0 - halo + x;
        if (n < 0 || n >= n_px) continue;
        if (su[x] <= mm) k = x;
    }
    double val;
    const int nk = m0 - halo + k;
    if (k < 0) {
        val = F[0];                                       // before the first moved point
    } else if (nk >= n_px - 1) {
        val = F[n_px - 1];                                // at or past the last moved point
    } else {
        const double w = expm1_small((mm - su[k]) * delta) / expm1_small((su[k + 1] - su[k]) * delta);
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
    const size_t tb = (size_t)n_rows * n_d * sizeof(double);
    const size_t off_o = (tb + 255) / 256 * 256;
    SOAP_TRY(ensure(c->bis_tab, off_o + (size_t)n_d * sizeof(double)));
    SOAP_TRY(upload_small(c, c->bis_tab.p, bis_host, tb));
    SOAP_TRY(upload_small(c, c->bis_tab.as<char>() + off_o, orig_host, (size_t)n_d * sizeof(double)));
    dim3 grid((unsigned)((c->n_px + kBisThreads - 1) / kBisThreads), (unsigned)n_rows);
    k_bisectors<<<grid, kBisThreads, 0, c->stream>>>(in, out, (int)c->n_px, n_d, c->bis_tab.as<double>(),
                                                     reinterpret_cast<const double*>(c->bis_tab.as<char>() + off_o),
                                                     1.0 / kCKms, 1.0 / c->delta, c->delta, halo, c->flags);
    SOAP_CUDA(cudaGetLastError());
    SOAP_LAUNCHED(c);
    return SOAP_OK;
}

}  // namespace soap
