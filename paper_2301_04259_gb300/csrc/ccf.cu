// ccf.cu -- G6: radial velocities from a line-mask CCF and a Gaussian fit (Sect. 4.1).
//
// Pixel n covers [n - 1/2, n + 1/2] in the pixel coordinate u = ln(lambda/lambda_s)/Delta.
// Mask line l at velocity v is a box of full width W centred at u_l + atanh(v/c)/Delta with
// half width h = W / (2 c Delta); CCF(v) = sum_l w_l sum_n F_n |pixel n intersect box|.
// Lines whose box leaves [-1/2, n_px - 1/2] anywhere on the velocity grid are skipped.
//
// k_ccf_partial: block = (chunk of 64 mask lines, block of spectra); thread = velocity.  The
// box position is computed in FP64 (it carries cm/s shifts), the overlaps and products in
// the spectra's precision; per-chunk partial sums are reduced in FP64 in a fixed order.
// k_gauss_fit: one warp per spectrum, FP64 Levenberg-Marquardt on
// A + B exp(-(v - mu)^2 / (2 s^2)).
#include <cmath>

#include "soap_internal.cuh"

namespace soap {

constexpr int kLinesPerChunk = 64;

__global__ void k_ccf_lines(int n_lines, const double* __restrict__ lam, double lam_s, double delta,
                            double h, double s_lo, double s_hi, int64_t n_px, double* u0h,
                            int* valid) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n_lines; l += gridDim.x * blockDim.x) {
        double u = log(lam[l] / lam_s) / delta;
        valid[l] = (u + s_lo - h >= -0.5) && (u + s_hi + h <= (double)n_px - 0.5);
        u0h[l] = u - h + 0.5;      // box start, shifted so that pixel n covers [n, n+1)
    }
}

template <typename T, int SB>
__global__ void k_ccf_partial(int n_lines, const double* __restrict__ u0h, const int* __restrict__ valid,
                              const double* __restrict__ weight, int n_v, double v_lo, double v_step,
                              double delta, double box, int64_t n_px, int n_spec,
                              const T* __restrict__ spectra, double* __restrict__ partial) {
    const int chunk = blockIdx.x;
    const int s0 = blockIdx.y * SB;
    const int l0 = chunk * kLinesPerChunk;
    const int l1 = min(n_lines, l0 + kLinesPerChunk);
    const int ns = min(SB, n_spec - s0);
    const T boxT = (T)box;
    for (int k = threadIdx.x; k < n_v; k += blockDim.x) {
        const double sk = atanh((v_lo + (double)k * v_step) / kCKms) / delta;
        T acc[SB];
#pragma unroll
        for (int s = 0; s < SB; s++) acc[s] = T(0);
        for (int l = l0; l < l1; l++) {
            if (!valid[l]) continue;
            const double t = u0h[l] + sk;
            const double fl = floor(t);
            const int64_t n0 = (int64_t)fl;
            const T phi = (T)(t - fl);
            const T wl = (T)weight[l];
            // overlap with pixel n0 + i: clamp(phi + box - i, 0, 1) for i >= 1, min(1-phi, box) for i = 0
            T ov = fmin(T(1) - phi, boxT);
            int i = 0;
            while (true) {
                const int64_t n = n0 + i;
                if (n >= n_px) break;                  // rounding at the grid edge only
                if (n >= 0) {
                    const T cwt = wl * ov;
                    const T* f = spectra + (int64_t)s0 * n_px + n;
#pragma unroll
                    for (int s = 0; s < SB; s++)
                        if (s < ns) acc[s] = fma(cwt, f[(int64_t)s * n_px], acc[s]);
                }
                i++;
                T rem = phi + boxT - (T)i;
                if (!(rem > T(0))) break;
                ov = fmin(rem, T(1));
            }
        }
        for (int s = 0; s < ns; s++)
            partial[((int64_t)chunk * n_spec + s0 + s) * n_v + k] = (double)acc[s];
    }
}

__global__ void k_ccf_reduce(int n_chunks, int n_spec, int n_v, const double* __restrict__ partial,
                             double* __restrict__ ccf) {
    const int64_t total = (int64_t)n_spec * n_v;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < n_chunks; c++) s += partial[(int64_t)c * total + t];
        ccf[t] = s;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Solve the 4x4 symmetric positive system M x = b by Gaussian elimination with partial
// pivoting (all lanes do it redundantly).
__device__ bool solve4(double M[4][4], double b[4], double x[4]) {
    for (int col = 0; col < 4; col++) {
        int piv = col;
        for (int r = col + 1; r < 4; r++)
            if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
        if (!(fabs(M[piv][col]) > 0.0)) return false;
        if (piv != col) {
            for (int q = 0; q < 4; q++) { double t = M[col][q]; M[col][q] = M[piv][q]; M[piv][q] = t; }
            double t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        for (int r = col + 1; r < 4; r++) {
            double f = M[r][col] / M[col][col];
            for (int q = col; q < 4; q++) M[r][q] -= f * M[col][q];
            b[r] -= f * b[col];
        }
    }
    for (int r = 3; r >= 0; r--) {
        double s = b[r];
        for (int q = r + 1; q < 4; q++) s -= M[r][q] * x[q];
        x[r] = s / M[r][r];
    }
    return true;
}

__device__ double model_cost(const double* __restrict__ c, int n_v, double v_lo, double v_step,
                             const double p[4], int lane) {
    double acc = 0.0;
    for (int k = lane; k < n_v; k += 32) {
        double v = v_lo + k * v_step;
        double z = (v - p[2]) / p[3];
        double r = p[0] + p[1] * exp(-0.5 * z * z) - c[k];
        acc += r * r;
    }
    return warp_sum(acc);
}

__global__ void k_gauss_fit(int n_spec, int n_v, double v_lo, double v_step,
                            const double* __restrict__ ccf, double* rv, double* fit) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_spec) return;
    const double* c = ccf + (int64_t)warp * n_v;
    // starting point: continuum = max, depth at the (first) minimum, width from the dip area
    double mx = -INFINITY, mn = INFINITY, sum = 0.0;
    int kmin = n_v;
    for (int k = lane; k < n_v; k += 32) {
        double v = c[k];
        mx = fmax(mx, v);
        sum += v;
        if (v < mn) { mn = v; kmin = k; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        double omn = __shfl_xor_sync(0xffffffffu, mn, o);
        int okm = __shfl_xor_sync(0xffffffffu, kmin, o);
        if (omn < mn || (omn == mn && okm < kmin)) { mn = omn; kmin = okm; }
    }
    sum = warp_sum(sum);
    double p[4];
    p[0] = mx;
    p[1] = mn - mx;
    p[2] = v_lo + kmin * v_step;
    double area = ((double)n_v * mx - sum) * v_step;
    double s0 = p[1] != 0.0 ? area / (fabs(p[1]) * sqrt(2.0 * kPi)) : v_step;
    p[3] = fmax(s0, v_step);
    double lam = 1e-3;
    double cost = model_cost(c, n_v, v_lo, v_step, p, lane);
    for (int it = 0; it < 400; it++) {
        double jtj[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, jtr[4] = {0, 0, 0, 0};
        for (int k = lane; k < n_v; k += 32) {
            double v = v_lo + k * v_step;
            double d = v - p[2];
            double e = exp(-0.5 * d * d / (p[3] * p[3]));
            double r = p[0] + p[1] * e - c[k];
            double J[4] = {1.0, e, p[1] * e * d / (p[3] * p[3]), p[1] * e * d * d / (p[3] * p[3] * p[3])};
            int q = 0;
            for (int a = 0; a < 4; a++) {
                jtr[a] += J[a] * r;
                for (int b = a; b < 4; b++) jtj[q++] += J[a] * J[b];
            }
        }
        for (int q = 0; q < 10; q++) jtj[q] = warp_sum(jtj[q]);
        for (int a = 0; a < 4; a++) jtr[a] = warp_sum(jtr[a]);
        bool accepted = false;
        double step_rel = 0.0;
        for (int tries = 0; tries < 40 && !accepted; tries++) {
            double M[4][4], b[4], dx[4];
            int q = 0;
            for (int a = 0; a < 4; a++)
                for (int bb = a; bb < 4; bb++) { M[a][bb] = M[bb][a] = jtj[q++]; }
            for (int a = 0; a < 4; a++) { M[a][a] *= (1.0 + lam); b[a] = -jtr[a]; }
            if (!solve4(M, b, dx)) { lam *= 10.0; continue; }
            double pn[4] = {p[0] + dx[0], p[1] + dx[1], p[2] + dx[2], p[3] + dx[3]};
            double cn = model_cost(c, n_v, v_lo, v_step, pn, lane);
            if (cn <= cost) {
                step_rel = 0.0;
                for (int a = 0; a < 4; a++)
                    step_rel = fmax(step_rel, fabs(dx[a]) / (fabs(p[a]) + 1e-300));
                for (int a = 0; a < 4; a++) p[a] = pn[a];
                cost = cn;
                lam = fmax(lam * 0.1, 1e-12);
                accepted = true;
            } else {
                lam *= 10.0;
            }
        }
        if (!accepted || step_rel < 1e-15) break;
    }
    if (lane == 0) {
        rv[warp] = p[2];
        if (fit) {
            fit[(int64_t)warp * 4 + 0] = p[0];
            fit[(int64_t)warp * 4 + 1] = p[1];
            fit[(int64_t)warp * 4 + 2] = p[2];
            fit[(int64_t)warp * 4 + 3] = fabs(p[3]);
        }
    }
}

soap_status rv_ccf_run(soap_ctx* c, const void* spectra_dev, int f32, int n_spec,
                       const double* mask_lambda, const double* mask_weight, int n_lines,
                       double width_kms, double v_lo, double v_step, int n_v, double* rv_dev,
                       double* fit_dev, double* ccf_dev) {
    const int n_chunks = (n_lines + kLinesPerChunk - 1) / kLinesPerChunk;
    // scratch: lines (lambda, weight, u0h, valid), partial sums, ccf
    size_t off_w = (size_t)n_lines * 8;
    size_t off_u = off_w + (size_t)n_lines * 8;
    size_t off_v = off_u + (size_t)n_lines * 8;
    size_t off_p = (off_v + (size_t)n_lines * 4 + 255) / 256 * 256;
    size_t off_c = off_p + (size_t)n_chunks * n_spec * n_v * 8;
    size_t total = off_c + (size_t)n_spec * n_v * 8;
    SOAP_TRY(ensure(c->ccf_tmp, total));
    char* base = c->ccf_tmp.as<char>();
    double* d_lam = (double*)base;
    double* d_w = (double*)(base + off_w);
    double* d_u = (double*)(base + off_u);
    int* d_valid = (int*)(base + off_v);
    double* d_part = (double*)(base + off_p);
    double* d_ccf = ccf_dev ? ccf_dev : (double*)(base + off_c);
    SOAP_CUDA(cudaMemcpyAsync(d_lam, mask_lambda, (size_t)n_lines * 8, cudaMemcpyHostToDevice, c->stream));
    SOAP_CUDA(cudaMemcpyAsync(d_w, mask_weight, (size_t)n_lines * 8, cudaMemcpyHostToDevice, c->stream));
    cudaEvent_t tb = c->profiling ? timer_begin(c) : nullptr;
    const double h = width_kms / (2.0 * kCKms * c->delta);
    const double v_hi = v_lo + v_step * (n_v - 1);
    k_ccf_lines<<<(n_lines + 255) / 256, 256, 0, c->stream>>>(
        n_lines, d_lam, c->lam_s, c->delta, h, std::atanh(v_lo / kCKms) / c->delta,
        std::atanh(v_hi / kCKms) / c->delta, c->n_px, d_u, d_valid);
    SOAP_LAUNCHED(c);
    const int threads = n_v >= 256 ? 256 : ((n_v + 31) / 32) * 32;
    if (f32) {
        constexpr int SB = 16;
        dim3 grid((unsigned)n_chunks, (unsigned)((n_spec + SB - 1) / SB));
        k_ccf_partial<float, SB><<<grid, threads, 0, c->stream>>>(
            n_lines, d_u, d_valid, d_w, n_v, v_lo, v_step, c->delta, 2.0 * h, c->n_px, n_spec,
            (const float*)spectra_dev, d_part);
    } else {
        constexpr int SB = 8;
        dim3 grid((unsigned)n_chunks, (unsigned)((n_spec + SB - 1) / SB));
        k_ccf_partial<double, SB><<<grid, threads, 0, c->stream>>>(
            n_lines, d_u, d_valid, d_w, n_v, v_lo, v_step, c->delta, 2.0 * h, c->n_px, n_spec,
            (const double*)spectra_dev, d_part);
    }
    SOAP_LAUNCHED(c);
    int64_t tot = (int64_t)n_spec * n_v;
    int g = (int)((tot + 255) / 256);
    if (g > 152 * 8) g = 152 * 8;
    k_ccf_reduce<<<g, 256, 0, c->stream>>>(n_chunks, n_spec, n_v, d_part, d_ccf);
    SOAP_LAUNCHED(c);
    if (c->profiling) timer_end(c, SOAP_TIMER_CCF, tb);
    int warps_per_block = 4;
    SOAP_TIMED(c, SOAP_TIMER_FIT,
               k_gauss_fit<<<(n_spec + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0,
                             c->stream>>>(n_spec, n_v, v_lo, v_step, d_ccf, rv_dev, fit_dev);
               SOAP_LAUNCHED(c));
    return SOAP_OK;
}

}  // namespace soap
