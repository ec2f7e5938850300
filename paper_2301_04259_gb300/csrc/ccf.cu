// ccf.cu -- G6: radial velocities from a line-mask CCF and a Gaussian fit (Sect. 4.1).
//
// Pixel n covers [n - 1/2, n + 1/2] in the pixel coordinate u = ln(lambda/lambda_s)/Delta.
// Mask line l at velocity v is a box of full width W centred at u_l + atanh(v/c)/Delta with
// half width h = W / (2 c Delta); CCF(v) = sum_l w_l sum_n F_n |pixel n intersect box|.
// Lines whose box leaves [-1/2, n_px - 1/2] anywhere on the velocity grid are skipped.
//
// Line and velocity tables (k_ccf_lines, k_ccf_velocities) split each box start into an integer
// pixel and an exact fraction (FP64: they carry cm/s shifts) and are kept while the mask and the
// velocity grid are unchanged.  Partial CCF sums per chunk of lines come from one of three
// kernels: k_ccf_tile (FP32 spectra, mask sorted by wavelength: register tiles of 4 velocities x
// 16 spectra per thread over staged pixel windows), k_ccf_window (FP64 spectra or boxes too wide
// for the tiles: staged windows, one velocity per thread) and k_ccf_partial (any line order).
// k_ccf_reduce adds the partials in a fixed order (FP64, or float pairs with TwoSum); k_gauss_fit
// fits A + B exp(-(v - mu)^2 / (2 s^2)) per spectrum (one block each: FP32 Levenberg-Marquardt,
// then Newton steps with FP64 residuals; see its comment).
#include <cmath>
#include <cstring>
#include <type_traits>
#include <algorithm>
#include <atomic>
#include <mutex>

#include "soap_internal.cuh"

namespace soap {

constexpr int kLinesPerChunk = 128;      // generic kernel
constexpr int kWinLines = 32;             // windowed kernel: 32 lines span ~600 px here
constexpr int kWinMax = 768;              // staged pixels per block (window budget)
constexpr int kReduceSplit = 8;

// Per line: validity and the box start a0 = u_l - h + 1/2 (pixel n covers [n, n+1) in a0 + s
// coordinates), split into an integer U_l and an exact fraction f_l in [0, 1).
__global__ void k_ccf_lines(int n_lines, const double* __restrict__ lam, const double* __restrict__ w,
                            double lam_s, double delta, double h, double s_lo, double s_hi,
                            int64_t n_px, int* U, double* f64, float* f32, float* w32, int* valid) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n_lines; l += gridDim.x * blockDim.x) {
        w32[l] = (float)w[l];
        double u = log(lam[l] / lam_s) / delta;
        valid[l] = (u + s_lo - h >= -0.5) && (u + s_hi + h <= (double)n_px - 0.5);
        double a0 = u - h + 0.5;
        double fl = floor(a0);
        U[l] = (int)fl;
        f64[l] = a0 - fl;
        f32[l] = (float)(a0 - fl);
    }
}

// Per velocity: s_k = atanh(v_k / c) / Delta split into an integer S_k and a fraction g_k.
__global__ void k_ccf_velocities(int n_v, double v_lo, double v_step, double delta, int* S,
                                 double* g64, float* g32) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_v; k += gridDim.x * blockDim.x) {
        double s = atanh((v_lo + (double)k * v_step) / kCKms) / delta;
        double fl = floor(s);
        S[k] = (int)fl;
        g64[k] = s - fl;
        g32[k] = (float)(s - fl);
    }
}

// Block = (chunk of lines, block of SB spectra); thread = velocity.  Box start in pixel units:
// (U_l + S_k) + (f_l + g_k); the fractional part carries the sub-pixel position in T.
template <typename T, int SB>
__global__ void k_ccf_partial(int n_lines, const int* __restrict__ U, const T* __restrict__ f,
                              const int* __restrict__ valid, const double* __restrict__ weight,
                              int n_v, const int* __restrict__ S, const T* __restrict__ g,
                              double box, int64_t n_px, int n_spec, const T* __restrict__ spectra,
                              double* __restrict__ partial) {
    const int chunk = blockIdx.x;
    const int s0 = blockIdx.y * SB;
    const int l0 = chunk * kLinesPerChunk;
    const int l1 = min(n_lines, l0 + kLinesPerChunk);
    const int ns = min(SB, n_spec - s0);
    const T boxT = (T)box;
    for (int k = threadIdx.x; k < n_v; k += blockDim.x) {
        const int Sk = S[k];
        const T gk = g[k];
        T acc[SB];
#pragma unroll
        for (int s = 0; s < SB; s++) acc[s] = T(0);
        for (int l = l0; l < l1; l++) {
            if (!valid[l]) continue;
            T fr = f[l] + gk;
            const int carry = fr >= T(1);
            const T phi = fr - (T)carry;
            const int64_t n0 = (int64_t)U[l] + Sk + carry;
            const T wl = (T)weight[l];
            // overlap with pixel n0 + i: min(1 - phi, box) for i = 0, clamp(phi + box - i, 0, 1) after
            T ov = fmin(T(1) - phi, boxT);
            int i = 0;
            while (true) {
                const int64_t n = n0 + i;
                if (n >= n_px) break;                  // rounding at the grid edge only
                if (n >= 0) {
                    const T cwt = wl * ov;
                    const T* fp = spectra + (int64_t)s0 * n_px + n;
#pragma unroll
                    for (int s = 0; s < SB; s++)
                        if (s < ns) acc[s] = fma(cwt, __ldg(fp + (int64_t)s * n_px), acc[s]);
                }
                i++;
                const T rem = phi + boxT - (T)i;
                if (!(rem > T(0))) break;
                ov = fmin(rem, T(1));
            }
        }
        for (int s = 0; s < ns; s++)
            partial[((int64_t)chunk * n_spec + s0 + s) * n_v + k] = (double)acc[s];
    }
}

// Windowed form for masks sorted by wavelength: the block stages the pixels its chunk of
// lines can reach, for its SB spectra, in shared memory as [pixel][SB] (one 16-byte vector per
// 4 spectra), so each overlap costs SB/4 vector loads instead of SB scattered global loads.
// Blocks whose window would not fit fall back to global loads.
// Windowed form for masks sorted by wavelength.  Block = (group of line chunks, SB spectra);
// thread = velocity k.  Per chunk the block stages the pixels its lines can reach, for its SB
// spectra, in shared memory as padded rows [pixel][SB] (one 16-byte vector per VW spectra).
// For each line the box position (integer pixel + fraction) is computed once and reused for
// all SB spectra; the box covers at most NB pixels, handled branch-free (zero overlaps add
// zero).  Chunks whose window does not fit fall back to global loads.
template <typename T, int SB, int NB>
__global__ void __launch_bounds__(256)
k_ccf_window(int n_lines, const int* __restrict__ U, const T* __restrict__ f,
             const int* __restrict__ valid, const T* __restrict__ wl_, int n_v,
             const int* __restrict__ S, const T* __restrict__ g, double box, int64_t n_px,
             int n_spec, const T* __restrict__ spectra, T* __restrict__ partial) {
    typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type V;
    constexpr int VW = sizeof(V) / sizeof(T);
    static_assert(SB % VW == 0, "SB must be a multiple of the vector width");
    constexpr int ROW = SB + 16 / (int)sizeof(T);         // padded row: consecutive rows on other banks
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int sB[kWinLines];                        // U_l - n_lo (window-relative base)
    __shared__ T sF[kWinLines];
    __shared__ T sW[kWinLines];
    T* win = reinterpret_cast<T*>(smraw);
    const int s0 = blockIdx.y * SB;
    const int ns = min(SB, n_spec - s0);
    const int n_chunks = (n_lines + kWinLines - 1) / kWinLines;
    const T boxT = (T)box;
    const int k = threadIdx.x;
    const bool active = k < n_v;
    const int Sk = active ? S[k] : 0;
    const T gk = active ? g[k] : T(0);
    T acc[SB];
#pragma unroll
    for (int s = 0; s < SB; s++) acc[s] = T(0);
    for (int chunk = blockIdx.x; chunk < n_chunks; chunk += gridDim.x) {
        const int l0 = chunk * kWinLines;
        const int l1 = min(n_lines, l0 + kWinLines);
        // window [n_lo, n_hi) with a margin on both sides; pixels off the grid stage as 0
        const int64_t n_lo = (int64_t)U[l0] + S[0] - 2;
        const int64_t n_hi = (int64_t)U[l1 - 1] + S[n_v - 1] + NB + 2;
        const int W = (int)(n_hi - n_lo);
        const bool staged = W >= NB && W <= kWinMax;
        __syncthreads();                                  // previous chunk done with the window
        for (int j = threadIdx.x; j < l1 - l0; j += blockDim.x) {
            const int l = l0 + j;
            sB[j] = (int)((int64_t)U[l] - n_lo);
            sF[j] = f[l];
            sW[j] = valid[l] ? wl_[l] : T(0);             // lines whose box leaves the grid: skipped
        }
        if (staged) {
            // one pixel per thread and step, all SB spectra at once (SB loads in flight)
            const T* base = spectra + (int64_t)s0 * n_px + n_lo;
            for (int x = threadIdx.x; x < W; x += blockDim.x) {
                const int64_t pix = n_lo + x;
                const bool on = pix >= 0 && pix < n_px;
                const T* col = base + x;
                T v[SB];
#pragma unroll
                for (int s = 0; s < SB; s++) {
                    v[s] = (on && s < ns) ? __ldg(col) : T(0);
                    col += n_px;
                }
                V* dst = reinterpret_cast<V*>(win + x * ROW);
#pragma unroll
                for (int q = 0; q < SB / VW; q++) {
                    V t;
                    if constexpr (VW == 4) t = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    else t = make_double2(v[2 * q], v[2 * q + 1]);
                    dst[q] = t;
                }
            }
        }
        __syncthreads();
        if (!active) continue;
        const int nl = l1 - l0;
        for (int j = 0; j < nl; j++) {
            const T wl = sW[j];
            if (wl == T(0)) continue;
            const T fr = sF[j] + gk;
            const bool carry = fr >= T(1);
            const T phi = carry ? fr - T(1) : fr;
            const int n = sB[j] + Sk + (carry ? 1 : 0);  // first pixel, window-relative
            const T end = phi + boxT;                      // box end measured from pixel n
            if (staged) {
                const int nc = min(max(n, 0), W - NB);   // always n itself (margins); kept for safety
#pragma unroll
                for (int i = 0; i < NB; i++) {
                    const T lo = i == 0 ? phi : T(i);
                    const T hi = end < T(i + 1) ? end : T(i + 1);
                    const T ov = hi > lo ? hi - lo : T(0);        // overlap of the box with pixel n + i
                    const T cwt = wl * ov;
                    const V* src = reinterpret_cast<const V*>(win + (nc + i) * ROW);
#pragma unroll
                    for (int q = 0; q < SB / VW; q++) {
                        const V t = src[q];
                        if constexpr (VW == 4) {
                            acc[4 * q] = fma(cwt, t.x, acc[4 * q]);
                            acc[4 * q + 1] = fma(cwt, t.y, acc[4 * q + 1]);
                            acc[4 * q + 2] = fma(cwt, t.z, acc[4 * q + 2]);
                            acc[4 * q + 3] = fma(cwt, t.w, acc[4 * q + 3]);
                        } else {
                            acc[2 * q] = fma(cwt, t.x, acc[2 * q]);
                            acc[2 * q + 1] = fma(cwt, t.y, acc[2 * q + 1]);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < NB; i++) {
                    const int64_t pix = n_lo + n + i;
                    if (pix < 0 || pix >= n_px) continue;
                    const T lo = i == 0 ? phi : T(i);
                    const T ov = fmax(fmin(end, T(i + 1)) - lo, T(0));
                    const T cwt = wl * ov;
                    const T* fp = spectra + (int64_t)s0 * n_px + pix;
#pragma unroll
                    for (int s = 0; s < SB; s++)
                        if (s < ns) acc[s] = fma(cwt, __ldg(fp + (int64_t)s * n_px), acc[s]);
                }
            }
        }
    }
    if (active)
        for (int s = 0; s < ns; s++)
            partial[((int64_t)blockIdx.x * n_spec + s0 + s) * n_v + k] = acc[s];   // FP64 in the reduction
}

// Register-tiled form for FP32 spectra and masks sorted by wavelength.  Block = (range of
// lines, kTileSB spectra); thread = (group of kTileVT consecutive velocities, line lane).  For a
// line, the boxes of a group's velocities start at a_kk = a_0 + (s_kk - s_k0) pixels from the
// group's first pixel n0 and, with the host's bound on the group's spread, all lie in the NP
// pixels n0 .. n0 + NP - 1.  Each of those pixels is read once from the staged window (all
// kTileSB spectra: four 16-byte loads) and applied to every velocity of the group with its
// overlap (zero where a box misses the pixel): NP x VT x SB FMAs per line for 4 x NP loads,
// against 2 x SB FMAs for 2 x 4 loads per velocity when a thread owns one velocity (the FMAs of
// spectrum pairs as two-wide fma.rn.f32x2).  The line
// lanes take alternate lines of each window; their sums are added in lane order at the end.
// Lines are staged kTileCL at a time in windows of at most kTileWin pixels (a window closes
// early where the lines spread out), so every line is handled in shared memory.
// Two-wide FP32 arithmetic on 64-bit register pairs (sm_100 and later): fma.rn.f32x2 performs two
// independent IEEE single-precision FMAs, so results equal those of two fmaf calls.
__device__ __forceinline__ unsigned long long f32x2_dup(float x) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ unsigned long long f32x2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f32x2_unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ void f32x2_fma(unsigned long long& d, unsigned long long a, unsigned long long b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

constexpr int kTileVT = 4;
constexpr int kTileSB = 16;
constexpr int kTileLP = 2;
constexpr int kTileCL = 16;
constexpr int kTileWin = 320;
constexpr int kTileRow = kTileSB + 2;                           // padded row (floats)
constexpr int kTileRed = kTileVT * kTileSB + 1;                 // lane-sum row (floats, padded)
constexpr int kTileMaxGroups = kTileWin * kTileRow / kTileRed;  // lane sums reuse the window
static_assert(kTileLP == 2, "the lane sums below add exactly two lanes");

template <int NP, int SB, bool SKIP0>
__global__ void __launch_bounds__(256)
k_ccf_tile(int n_lines, int lines_per_block, const int* __restrict__ U, const float* __restrict__ f,
           const int* __restrict__ valid, const float* __restrict__ wl_, int n_v,
           const int* __restrict__ S, const float* __restrict__ g, float box, int64_t n_px,
           int n_spec, int s_base, const float* __restrict__ spectra, float* __restrict__ partial) {
    static_assert(SB % 4 == 0 && SB <= kTileSB, "SB: a multiple of 4, at most kTileSB");
    // Row pitch SB + 2 floats, read as 8-byte pairs: for 16 spectra a row is 9 pairs, so the
    // rows a half-warp reads (16 velocity groups, about 1.2 pixels apart) fall on distinct
    // banks unless 16 rows apart
    constexpr int ROW = SB + 2;
    constexpr int RED = kTileVT * SB + 1;                  // lane-sum row (floats, padded)
    __shared__ __align__(16) float win[kTileWin * kTileRow];
    __shared__ int sB[kTileCL];
    __shared__ float sF[kTileCL];
    __shared__ float sW[kTileCL];
    // velocity groups padded to a multiple of 16, so no half-warp mixes the two line lanes
    const int NG = (n_v + kTileVT - 1) / kTileVT;
    const int NGP = (NG + 15) & ~15;
    const int lane = threadIdx.x / NGP;
    const int gi = threadIdx.x - lane * NGP;
    const bool active = lane < kTileLP && gi < NG;
    const int k0 = gi * kTileVT;
    const int s0 = s_base + blockIdx.y * SB;
    const int ns = min(SB, n_spec - s0);
    const int L0 = blockIdx.x * lines_per_block;
    const int L1 = min(n_lines, L0 + lines_per_block);
    int S0 = 0;
    float g0 = 0.0f;
    float rel[kTileVT];
#pragma unroll
    for (int kk = 0; kk < kTileVT; kk++) rel[kk] = 0.0f;
    if (active) {
        S0 = S[k0];
        g0 = g[k0];
#pragma unroll
        for (int kk = 0; kk < kTileVT; kk++) {
            const int k = min(k0 + kk, n_v - 1);          // past the grid: a copy of the last
            rel[kk] = (float)(S[k] - S0) + g[k];
        }
    }
    const int Smin = S[0], sweep = S[n_v - 1] - Smin;
    const int budget = kTileWin - sweep - NP - 5;           // >= 0 (checked by the host)
    // accumulators of spectrum pairs (2i, 2i+1) share a 64-bit register: one two-wide FMA
    // (fma.rn.f32x2, two independent IEEE FMAs) per pair
    unsigned long long acc[kTileVT][SB / 2];
#pragma unroll
    for (int kk = 0; kk < kTileVT; kk++)
#pragma unroll
        for (int s = 0; s < SB / 2; s++) acc[kk][s] = 0ull;
    const float* base = spectra + (int64_t)s0 * n_px;
    for (int j0 = L0; j0 < L1;) {
        // lines j0 .. j1-1 whose boxes fit one window
        const int Ub = U[j0];
        int Umax = Ub, j1 = j0 + 1;
        while (j1 < L1 && j1 - j0 < kTileCL) {
            const int u = U[j1];
            if (u - Ub > budget) break;
            Umax = max(Umax, u);
            j1++;
        }
        const int64_t n_lo = (int64_t)Ub + Smin - 2;
        const int W = (Umax - Ub) + sweep + NP + 5;          // <= kTileWin
        __syncthreads();                                   // the previous window is consumed
        for (int j = threadIdx.x; j < j1 - j0; j += blockDim.x) {
            sB[j] = (int)((int64_t)U[j0 + j] - n_lo);
            sF[j] = f[j0 + j];
            sW[j] = valid[j0 + j] ? wl_[j0 + j] : 0.0f;     // lines whose box leaves the grid: skipped
        }
        for (int x = threadIdx.x; x < W; x += blockDim.x) {
            const int64_t pix = n_lo + x;
            const bool on = pix >= 0 && pix < n_px;
            const float* col = base + pix;                  // spectrum s at col + s n_px (added, not multiplied)
            float v[SB];
#pragma unroll
            for (int s = 0; s < SB; s++) {
                v[s] = (on && s < ns) ? __ldg(col) : 0.0f;
                col += n_px;
            }
            float2* dst = reinterpret_cast<float2*>(win + x * ROW);
#pragma unroll
            for (int q = 0; q < SB / 2; q++) dst[q] = make_float2(v[2 * q], v[2 * q + 1]);
        }
        __syncthreads();
        if (active) {
            for (int j = lane; j < j1 - j0; j += kTileLP) {
                const float wl = sW[j];
                if (wl == 0.0f) continue;
                const float fl = sF[j];
                const bool carry = fl + g0 >= 1.0f;
                const float cf = carry ? 1.0f : 0.0f;
                const int n0 = sB[j] + S0 + (carry ? 1 : 0);
                // overlap of box [a, e) with pixel n0 + jj: sat(e - jj) - sat(a - jj) (sat: clamp
                // to [0, 1]; x - jj is exact for the small box coordinates here), times w_l
                unsigned long long ov[kTileVT][NP];
#pragma unroll
                for (int kk = 0; kk < kTileVT; kk++) {
                    const float a = (fl + rel[kk]) - cf;     // box start from pixel n0
                    const float e = a + box;
#pragma unroll
                    for (int jj = 0; jj < NP; jj++) {
                        const float o = (SKIP0 && kk == 0 && jj >= 2)
                                            ? 0.0f
                                            : wl * (__saturatef(e - (float)jj) - __saturatef(a - (float)jj));
                        ov[kk][jj] = f32x2_dup(o);
                    }
                }
#pragma unroll
                for (int jj = 0; jj < NP; jj++) {
                    const float2* src = reinterpret_cast<const float2*>(win + (n0 + jj) * ROW);
                    unsigned long long t[SB / 2];
#pragma unroll
                    for (int q = 0; q < SB / 2; q++) {
                        const float2 x = src[q];
                        t[q] = f32x2_pack(x.x, x.y);
                    }
#pragma unroll
                    for (int kk = 0; kk < kTileVT; kk++) {
                        // the first velocity's box starts in pixel n0: one no wider than a pixel
                        // ends before pixel n0 + 2
                        if (SKIP0 && kk == 0 && jj >= 2) continue;
#pragma unroll
                        for (int s = 0; s < SB / 2; s++) f32x2_fma(acc[kk][s], ov[kk][jj], t[s]);
                    }
                }
            }
        }
        j0 = j1;
    }
    // lane sums in lane order (lane 1 through shared memory), one partial row per block
    __syncthreads();
    if (active && lane == 1)
#pragma unroll
        for (int kk = 0; kk < kTileVT; kk++)
#pragma unroll
            for (int s = 0; s < SB / 2; s++)
                f32x2_unpack(acc[kk][s], win[gi * RED + kk * SB + 2 * s], win[gi * RED + kk * SB + 2 * s + 1]);
    __syncthreads();
    if (active && lane == 0) {
#pragma unroll
        for (int kk = 0; kk < kTileVT; kk++) {
            const int k = k0 + kk;
            if (k >= n_v) break;
#pragma unroll
            for (int s = 0; s < SB / 2; s++) {
                float lo, hi;
                f32x2_unpack(acc[kk][s], lo, hi);
                if (2 * s < ns)
                    partial[((int64_t)blockIdx.x * n_spec + s0 + 2 * s) * n_v + k] = lo + win[gi * RED + kk * SB + 2 * s];
                if (2 * s + 1 < ns)
                    partial[((int64_t)blockIdx.x * n_spec + s0 + 2 * s + 1) * n_v + k] =
                        hi + win[gi * RED + kk * SB + 2 * s + 1];
            }
        }
    }
}

// ccf[t] = sum over chunks of partial[c][t], in a fixed order: kReduceSplit threads take
// interleaved chunks, then a fixed tree adds their sums.  FP64 partials are added in
// FP64.  FP32 partials are added as unevaluated pairs hi + lo of floats with the error-free
// transformation TwoSum (Knuth): the pair carries ~48 bits, so the sum is as exact as an FP64
// sum of the same floats while every operation stays on the FP32 pipe (FP64 and float->double
// conversions run at 1/64 rate on this GPU); only the final pair is converted.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += x
__device__ __forceinline__ void pair_add(float& hi, float& lo, float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
}

// Block (32, kReduceSplit): lane x of warp y takes output t = 32 blockIdx.x + x and chunks y,
// y + kReduceSplit, ..., so each load instruction reads 32 consecutive outputs of one chunk
// (whole sectors; with the split across the lanes of a warp every load touched 32 sectors for 128
// useful bytes); the kReduceSplit sums of an output are then combined through shared memory by
// the fixed tree of the lane version (y += y + 4, y += y + 2, y += y + 1): the same results.
template <typename TP>
__global__ void __launch_bounds__(32 * kReduceSplit)
k_ccf_reduce(int n_chunks, int n_spec, int n_v, const TP* __restrict__ partial, double* __restrict__ ccf) {
    // launched early after the tensor-core CCF: wait for its partials, then let the fit start early
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int64_t total = (int64_t)n_spec * n_v;
    const int x = threadIdx.x, sub = threadIdx.y;
    const int64_t t = (int64_t)blockIdx.x * 32 + x;
    if constexpr (sizeof(TP) == 8) {
        __shared__ double sh[kReduceSplit][32];
        double s = 0.0;
        if (t < total) {
#pragma unroll 4
            for (int c = sub; c < n_chunks; c += kReduceSplit) s += (double)partial[(int64_t)c * total + t];
        }
        sh[sub][x] = s;
        __syncthreads();
        for (int o = kReduceSplit / 2; o > 0; o >>= 1) {
            if (sub < o) sh[sub][x] += sh[sub + o][x];
            __syncthreads();
        }
        if (sub == 0 && t < total) ccf[t] = sh[0][x];
    } else {
        __shared__ float shh[kReduceSplit][32], shl[kReduceSplit][32];
        float hi = 0.0f, lo = 0.0f;
        if (t < total) {
#pragma unroll 4
            for (int c = sub; c < n_chunks; c += kReduceSplit) pair_add(hi, lo, partial[(int64_t)c * total + t]);
        }
        shh[sub][x] = hi;
        shl[sub][x] = lo;
        __syncthreads();
        for (int o = kReduceSplit / 2; o > 0; o >>= 1) {
            if (sub < o) {
                float h = shh[sub][x], l = shl[sub][x];
                pair_add(h, l, shh[sub + o][x]);
                shh[sub][x] = h;
                shl[sub][x] = l + shl[sub + o][x];
            }
            __syncthreads();
        }
        if (sub == 0 && t < total) ccf[t] = (double)shh[0][x] + (double)shl[0][x];
    }
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Solve the 4x4 system M x = b by Gaussian elimination with partial pivoting (FP32).
__device__ bool solve4f(float M[4][4], float b[4], float x[4]) {
    for (int col = 0; col < 4; col++) {
        int piv = col;
        for (int r = col + 1; r < 4; r++)
            if (fabsf(M[r][col]) > fabsf(M[piv][col])) piv = r;
        if (!(fabsf(M[piv][col]) > 0.0f)) return false;
        if (piv != col) {
            for (int q = 0; q < 4; q++) { float t = M[col][q]; M[col][q] = M[piv][q]; M[piv][q] = t; }
            float t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        const float inv = 1.0f / M[col][col];
        for (int r = col + 1; r < 4; r++) {
            float f = M[r][col] * inv;
            for (int q = col; q < 4; q++) M[r][q] -= f * M[col][q];
            b[r] -= f * b[col];
        }
    }
    for (int r = 3; r >= 0; r--) {
        float s = b[r];
        for (int q = r + 1; q < 4; q++) s -= M[r][q] * x[q];
        x[r] = s / M[r][r];
    }
    return isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]) && isfinite(x[3]);
}

constexpr int kFitThreads = 128;
constexpr int kFitWarps = kFitThreads / 32;
constexpr int kFitCache = 4;            // velocities cached in registers per thread
constexpr int kFitPassesA = 80;         // FP32 Levenberg-Marquardt passes at most
constexpr int kFitPassesB = 8;          // Newton passes at most
constexpr float kFitTolA = 1e-4f;       // scaled step at which the FP32 phase hands over
constexpr float kFitTolB = 1e-6f;       // scaled Newton step after which one more step is exact

// Column sums of a [kFitThreads][NV] shared table in a fixed order: NV x 8 threads add 16 rows
// each, then NV threads add the 8 partial sums.  Thread 0 returns the totals in out.
template <int NV>
__device__ __forceinline__ void table_sum(const double (&v)[NV], double* tab, double* part,
                                          double (&out)[NV]) {
#pragma unroll
    for (int q = 0; q < NV; q++) tab[threadIdx.x * NV + q] = v[q];
    __syncthreads();
    if (threadIdx.x < NV * 8) {
        const int q = threadIdx.x % NV, seg = threadIdx.x / NV;
        double s = 0.0;
        for (int r = seg * (kFitThreads / 8); r < (seg + 1) * (kFitThreads / 8); r++) s += tab[r * NV + q];
        part[seg * NV + q] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int seg = 0; seg < 8; seg++) s += part[seg * NV + threadIdx.x];
        part[8 * NV + threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NV; q++) out[q] = part[8 * NV + q];
}

// Block-wide sums of NF floats and ND doubles that come out bit-identical in every thread: a
// xor butterfly inside each warp (addition commutes, so every lane ends with the same warp
// total), one shared row per warp, then the rows added in warp order.  Two buffers alternate,
// so one barrier per call suffices (a buffer is rewritten only after the next call's barrier).
constexpr int kSumF = 15, kSumD = 5;
template <int NF, int ND>
__device__ __forceinline__ void block_sums(float* f, double* d, float* sf, double* sd, int& buf) {
    static_assert(NF <= kSumF && ND <= kSumD, "shared rows too short");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < NF; q++) f[q] += __shfl_xor_sync(0xffffffffu, f[q], o);
#pragma unroll
        for (int q = 0; q < ND; q++) d[q] += __shfl_xor_sync(0xffffffffu, d[q], o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* rf = sf + buf * kFitWarps * kSumF;
    double* rd = sd + buf * kFitWarps * kSumD;
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NF; q++) rf[warp * kSumF + q] = f[q];
#pragma unroll
        for (int q = 0; q < ND; q++) rd[warp * kSumD + q] = d[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NF; q++) {
        float t = rf[q];
#pragma unroll
        for (int w = 1; w < kFitWarps; w++) t += rf[w * kSumF + q];
        f[q] = t;
    }
#pragma unroll
    for (int q = 0; q < ND; q++) {
        double t = rd[q];
#pragma unroll
        for (int w = 1; w < kFitWarps; w++) t += rd[w * kSumD + q];
        d[q] = t;
    }
    buf ^= 1;
}

// First phase, FP32: one pass at scaled parameters p = (a, b, m, w) of the model
// a + b exp(-(u - m)^2 / (2 w^2)) against y.  Returns in every thread the sums J^T J (10, upper
// triangle by rows), J^T r (4) and r^2.  uc / yc hold this thread's first kFitCache abscissae
// and ordinates; further points are read from y.
__device__ __forceinline__ void pass_a(const float p[4], int n_v, const float (&uc)[kFitCache],
                                       const float (&yc)[kFitCache], const double* __restrict__ y,
                                       float u0, float du, float* sf, double* sd, int& buf,
                                       float (&acc)[15]) {
#pragma unroll
    for (int q = 0; q < 15; q++) acc[q] = 0.0f;
    const float iw = 1.0f / p[3];
    const float iw2 = iw * iw;
    auto point = [&](float u, float yk) {
        const float d = u - p[2];
        const float e = expf(-0.5f * d * d * iw2);
        const float r = fmaf(p[1], e, p[0]) - yk;
        const float t = p[1] * e * d * iw2;
        const float J[4] = {1.0f, e, t, t * d * iw};
        int q = 0;
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = a; b < 4; b++) { acc[q] = fmaf(J[a], J[b], acc[q]); q++; }
#pragma unroll
        for (int a = 0; a < 4; a++) acc[10 + a] = fmaf(J[a], r, acc[10 + a]);
        acc[14] = fmaf(r, r, acc[14]);
    };
#pragma unroll
    for (int i = 0; i < kFitCache; i++)
        if (threadIdx.x + i * kFitThreads < n_v) point(uc[i], yc[i]);
    for (int k = threadIdx.x + kFitCache * kFitThreads; k < n_v; k += kFitThreads)
        point(fmaf((float)k, du, u0), (float)y[k]);
    block_sums<15, 0>(acc, nullptr, sf, sd, buf);
}

// Second phase: one Newton pass at p (FP64).  The residuals, the cost and the gradient J^T r
// are FP64 (they fix where the iteration stops); J^T J (10) and the residual-weighted sums
// R_j = sum r g d^j, j = 0..4 (g the Gaussian, d = u - m), which enter the Hessian
// H = J^T J + sum r d2m only as the step's metric, are FP32.  Returns f = (J^T J, R_0..R_4)
// and g = (J^T r, r^2) in every thread.
__device__ __forceinline__ void pass_b(const double p[4], int n_v, const double* __restrict__ y,
                                       double u0, double du, float* sf, double* sd, int& buf,
                                       float (&f)[15], double (&g)[5]) {
#pragma unroll
    for (int q = 0; q < 15; q++) f[q] = 0.0f;
#pragma unroll
    for (int q = 0; q < 5; q++) g[q] = 0.0;
    const double iw = 1.0 / p[3];
    const double iw2 = iw * iw;
    const float iwf = (float)iw;
    for (int k = threadIdx.x; k < n_v; k += kFitThreads) {
        const double d = fma((double)k, du, u0) - p[2];
        const double e = exp(-0.5 * d * d * iw2);
        const double r = fma(p[1], e, p[0]) - y[k];
        const double t = p[1] * e * d * iw2;
        g[0] += r;
        g[1] = fma(e, r, g[1]);
        g[2] = fma(t, r, g[2]);
        g[3] = fma(t * d * iw, r, g[3]);
        g[4] = fma(r, r, g[4]);
        const float ef = (float)e, df = (float)d, rf = (float)r, tf = (float)t;
        const float J[4] = {1.0f, ef, tf, tf * df * iwf};
        int q = 0;
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = a; b < 4; b++) { f[q] = fmaf(J[a], J[b], f[q]); q++; }
        float w = rf * ef;
#pragma unroll
        for (int j = 0; j < 5; j++) { f[10 + j] += w; w *= df; }
    }
    block_sums<15, 5>(f, g, sf, sd, buf);
}

// Upper-triangle index of (a, b), a <= b, in the 10 sums of J^T J.
__device__ __forceinline__ int tri(int a, int b) { return a * 4 - a * (a - 1) / 2 + (b - a); }

// One block of 128 threads per spectrum.  Start (as the oracle's): continuum A = max CCF,
// depth B = min - max at the (first) minimum, mu = its velocity, sigma from the dip's area.
// The fit runs in scaled variables (CCF / max, (v - mu0) / sigma0), model
// a + b exp(-(u - m)^2 / (2 w^2)), and ends at the least-squares minimum in two phases:
//  1. Levenberg-Marquardt in FP32 (damping J^T J + lam diag(J^T J)): a trial point is kept
//     when its cost does not grow (lam / 10, down to 1e-9), else dropped (lam x 10); the phase
//     ends once a step is below 1e-4 (relative for the amplitudes), lam passes 1e8, or after
//     kFitPassesA passes.  It only has to land in the basin of the minimum.
//  2. Newton steps on H = J^T J + sum r d2m with FP64 residuals and gradient: near the minimum
//     they converge quadratically (Gauss-Newton converges only linearly when, as for a
//     rotation-broadened CCF, the residuals are large), so once a step is below 1e-6 the
//     next one would be below rounding and the iteration stops after taking it.  A step is
//     taken only while it points downhill and the steps shrink; the cost may not grow by more
//     than 1e-12 relative from one pass to the next (else the previous point is kept).
// Every thread runs the same iteration on bit-identical sums, so no broadcast is needed.
// win (nullable): per spectrum, the first velocity index k0 and the number of points n of its
// fit window; the fit then sees the CCF at v_lo + (k0 + k) v_step, k = 0 .. n-1, only.
__global__ void __launch_bounds__(kFitThreads) k_gauss_fit(int n_spec, int n_v_grid, double v_lo_grid,
                                                           double v_step,
                                                           const double* __restrict__ ccf,
                                                           double* scratch, double* rv,
                                                           double* fit, const int* __restrict__ win) {
    __shared__ double tab[kFitThreads];
    __shared__ double part[9];
    __shared__ double red[kFitWarps][2];
    __shared__ int redk[kFitWarps];
    __shared__ double sp[2];
    __shared__ float sf[2 * kFitWarps * kSumF];
    __shared__ double sd[2 * kFitWarps * kSumD];
    const int spec = blockIdx.x;
    if (spec >= n_spec) return;
    int k0 = 0, n_v = n_v_grid;
    if (win) {
        k0 = win[2 * spec];
        n_v = win[2 * spec + 1];
    }
    const double v_lo = win ? fma((double)k0, v_step, v_lo_grid) : v_lo_grid;
    const double* c = ccf + (int64_t)spec * n_v_grid + k0;
    double* y = scratch + (int64_t)spec * n_v_grid + k0;  // scaled CCF
    double mx = -INFINITY, mn = INFINITY;
    int kmin = n_v;
    for (int k = threadIdx.x; k < n_v; k += kFitThreads) {
        mx = fmax(mx, c[k]);
        if (c[k] < mn) { mn = c[k]; kmin = k; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const double mo = __shfl_xor_sync(0xffffffffu, mn, o);
        const int ko = __shfl_xor_sync(0xffffffffu, kmin, o);
        if (mo < mn || (mo == mn && ko < kmin)) { mn = mo; kmin = ko; }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[warp][0] = mx; red[warp][1] = mn; redk[warp] = kmin; }
    __syncthreads();
    mx = red[0][0]; mn = red[0][1]; kmin = redk[0];
    for (int w = 1; w < kFitWarps; w++) {
        mx = fmax(mx, red[w][0]);
        if (red[w][1] < mn || (red[w][1] == mn && redk[w] < kmin)) { mn = red[w][1]; kmin = redk[w]; }
    }
    const double scale = mx != 0.0 ? fabs(mx) : 1.0;
    const double iscale = 1.0 / scale;
    double m1[1] = {0.0};
    for (int k = threadIdx.x; k < n_v; k += kFitThreads) {
        y[k] = c[k] * iscale;
        m1[0] += mx - c[k];
    }
    double area[1];
    table_sum<1>(m1, tab, part, area);
    if (threadIdx.x == 0) {
        const double B0 = mn - mx;
        const double s = B0 != 0.0 ? area[0] * v_step / (fabs(B0) * 2.5066282746310002) : v_step;
        sp[0] = fma((double)kmin, v_step, v_lo);
        sp[1] = fmax(s, v_step);
    }
    __syncthreads();
    const double c0 = sp[0], s0 = sp[1];
    const double u0 = (v_lo - c0) / s0, du = v_step / s0;
    float uc[kFitCache], yc[kFitCache];
#pragma unroll
    for (int i = 0; i < kFitCache; i++) {
        const int k = threadIdx.x + i * kFitThreads;
        uc[i] = k < n_v ? (float)fma((double)k, du, u0) : 0.0f;
        yc[i] = k < n_v ? (float)(c[k] * iscale) : 0.0f;
    }
    int buf = 0;

    // ---- phase 1: FP32 Levenberg-Marquardt ----
    float p[4] = {(float)(mx * iscale), (float)((mn - mx) * iscale), 0.0f, 1.0f};
    float pt[4] = {p[0], p[1], p[2], p[3]};
    float acc[15], jtj[10], jtr[4], cost = 0.0f, lam = 1e-3f;
    bool tiny = false;
    pass_a(p, n_v, uc, yc, y, (float)u0, (float)du, sf, sd, buf, acc);
    for (int it = 0; it < kFitPassesA; it++) {
        bool stop = false;
        if (it == 0 || acc[14] <= cost) {            // keep the trial point
            for (int a = 0; a < 4; a++) p[a] = pt[a];
            for (int q = 0; q < 10; q++) jtj[q] = acc[q];
            for (int a = 0; a < 4; a++) jtr[a] = acc[10 + a];
            cost = acc[14];
            if (it > 0) lam = fmaxf(lam * 0.1f, 1e-9f);
            if (tiny) stop = true;
        } else {
            if (tiny) stop = true;
            lam *= 10.0f;
        }
        while (!stop) {
            if (lam > 1e8f) { stop = true; break; }
            float M[4][4], b[4], dx[4];
            for (int a = 0; a < 4; a++)
                for (int bb = a; bb < 4; bb++) M[a][bb] = M[bb][a] = jtj[tri(a, bb)];
            for (int a = 0; a < 4; a++) { M[a][a] *= 1.0f + lam; b[a] = -jtr[a]; }
            if (!solve4f(M, b, dx)) { lam *= 10.0f; continue; }
            tiny = fabsf(dx[2]) <= kFitTolA && fabsf(dx[3]) <= kFitTolA &&
                   fabsf(dx[0]) <= kFitTolA * fabsf(p[0]) && fabsf(dx[1]) <= kFitTolA * fabsf(p[1]);
            for (int a = 0; a < 4; a++) pt[a] = p[a] + dx[a];
            break;
        }
        if (stop) break;
        pass_a(pt, n_v, uc, yc, y, (float)u0, (float)du, sf, sd, buf, acc);
    }

    // ---- phase 2: Newton with FP64 residuals ----
    double pd[4] = {p[0], p[1], p[2], p[3]};
    double prev[4] = {pd[0], pd[1], pd[2], pd[3]};
    double cost_prev = INFINITY;
    float last = INFINITY;
    for (int it = 0; it < kFitPassesB; it++) {
        float f[15];
        double g[5];
        pass_b(pd, n_v, y, u0, du, sf, sd, buf, f, g);
        if (!(g[4] <= cost_prev * (1.0 + 1e-12))) {   // the last step did not help: undo it
            for (int a = 0; a < 4; a++) pd[a] = prev[a];
            break;
        }
        const float b = (float)pd[1], w = (float)pd[3];
        const float iw = 1.0f / w, iw2 = iw * iw;
        const float R0 = f[10], R1 = f[11], R2 = f[12], R3 = f[13], R4 = f[14];
        float M[4][4], rhs[4], dx[4];
        for (int a = 0; a < 4; a++)
            for (int bb = a; bb < 4; bb++) M[a][bb] = M[bb][a] = f[tri(a, bb)];
        M[1][2] += R1 * iw2;
        M[1][3] += R2 * iw2 * iw;
        M[2][2] += b * iw2 * (R2 * iw2 - R0);
        M[2][3] += b * iw2 * iw * (R3 * iw2 - 2.0f * R1);
        M[3][3] += b * iw2 * iw2 * (R4 * iw2 - 3.0f * R2);
        M[2][1] = M[1][2];
        M[3][1] = M[1][3];
        M[3][2] = M[2][3];
        for (int a = 0; a < 4; a++) rhs[a] = -(float)g[a];
        if (!solve4f(M, rhs, dx)) break;
        if (!(dx[0] * rhs[0] + dx[1] * rhs[1] + dx[2] * rhs[2] + dx[3] * rhs[3] > 0.0f)) break;
        const float ref = fabsf((float)pd[0]), wref = fabsf(w);
        const float size = fmaxf(fmaxf(fabsf(dx[0]) / ref, fabsf(dx[1]) / ref),
                                 fmaxf(fabsf(dx[2]) / wref, fabsf(dx[3]) / wref));
        if (!(size < last)) break;
        for (int a = 0; a < 4; a++) { prev[a] = pd[a]; pd[a] += (double)dx[a]; }
        cost_prev = g[4];
        last = size;
        if (size <= kFitTolB) break;
    }

    if (threadIdx.x == 0) {
        // a fit that leaves the velocity grid (no dip to fit) is reported as NaN
        const double v_hi = fma((double)(n_v - 1), v_step, v_lo);
        double mu = fma(pd[2], s0, c0);
        if (!(mu >= v_lo && mu <= v_hi) || !(fabs(pd[3]) * s0 <= v_hi - v_lo)) mu = NAN;
        rv[spec] = mu;
        if (fit) {
            fit[(int64_t)spec * 4 + 0] = pd[0] * scale;
            fit[(int64_t)spec * 4 + 1] = pd[1] * scale;
            fit[(int64_t)spec * 4 + 2] = mu;
            fit[(int64_t)spec * 4 + 3] = fabs(pd[3]) * s0;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Gaussian fit of CCFs from float32 spectra: SPAN warps per spectrum, FP32 throughout.
// ---------------------------------------------------------------------------------------
// Such a CCF carries FP32 rounding (~1e-7 relative) already, so the fit needs no FP64: the
// FP32 residuals r = a + b e - y (|r| error ~1e-7 of the continuum) move the least-squares centre
// by ~1e-8 of the width, far below the mixed path's 1 cm/s.  The start, the scaled variables and
// the two phases are those of k_gauss_fit; the second phase is Newton on the exact Hessian in
// FP32.  A block has 4 warps: SPAN = 4 gives each spectrum the whole block (a short chain per
// pass: few spectra finish sooner), SPAN = 1 one warp (every lane repeats the small solves once
// per spectrum instead of four times: many spectra finish sooner).  Thread t of a spectrum takes
// the points k = t + 32 SPAN i; a pass's sums are warp xor butterflies, then (SPAN = 4) the
// warps' sums are added in warp order through shared memory, so every thread holds the same bits
// and runs the same iteration (the block's barriers are reached by all of its threads).  Points
// with i < Fw<SPAN>::cache stay in registers; further ones (more than 256 velocities) are kept as
// floats in the scratch row, each read back by the thread that wrote it.
template <int SPAN>
struct Fw {
    static_assert(SPAN == 1 || SPAN == 4, "one warp or the whole block per spectrum");
    static constexpr int threads = 32 * SPAN;                  // per spectrum
    static constexpr int cache = (256 + threads - 1) / threads;
    static constexpr int per_block = 4 / SPAN;                 // spectra per block of 4 warps
};
constexpr int kFwBlock = 128;
constexpr int kFwPassesA = 80;          // FP32 Levenberg-Marquardt passes at most
constexpr int kFwPassesB = 8;           // Newton passes at most
constexpr float kFwTolA = 1e-4f;        // scaled step at which Levenberg-Marquardt hands over
constexpr float kFwTolB = 2e-6f;        // scaled Newton step at FP32's resolution of the minimum
constexpr int kFwMaxSums = 20;

template <int NF>
__device__ __forceinline__ void warp_allsum(float (&f)[NF]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < NF; q++) f[q] += __shfl_xor_sync(0xffffffffu, f[q], o);
}

// Sums over a spectrum's threads, identical in every thread: warp butterflies, then the SPAN warp
// sums added in warp order.  buf: 2 x SPAN x kFwMaxSums floats, used alternately (a buffer is written
// again only after the next call's barrier, when every thread has read it).
template <int SPAN, int NF>
__device__ __forceinline__ void block_allsum(float (&f)[NF], float* buf, int& parity) {
    warp_allsum<NF>(f);
    if constexpr (SPAN > 1) {
        float* b = buf + parity * (SPAN * kFwMaxSums);
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int q = 0; q < NF; q++) b[w * kFwMaxSums + q] = f[q];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NF; q++) {
            float t = b[q];
#pragma unroll
            for (int v = 1; v < SPAN; v++) t += b[v * kFwMaxSums + q];
            f[q] = t;
        }
        parity ^= 1;
    }
}

// One pass at scaled parameters p of a + b exp(-(u - m)^2 / (2 w^2)): J^T J (10, upper
// triangle by rows), J^T r (4), r^2 (1) and, with HESS, R_j = sum r g d^j, j = 0..4 (g the
// Gaussian, d = u - m) for the second-derivative part of the Hessian.  u_k = (k - kmin) du.
template <int SPAN, bool HESS>
__device__ __forceinline__ void fw_pass(const float p[4], int n_v, int kmin, float du, int t,
                                        const float (&yc)[Fw<SPAN>::cache], const float* __restrict__ ys,
                                        float (&acc)[HESS ? 20 : 15], float* buf, int& parity) {
    constexpr int kFwThreads = Fw<SPAN>::threads, kFwCache = Fw<SPAN>::cache;
    constexpr int NF = HESS ? 20 : 15;
#pragma unroll
    for (int q = 0; q < NF; q++) acc[q] = 0.0f;
    const float iw = 1.0f / p[3];
    const float iw2 = iw * iw;
    auto point = [&](int k, float yk) {
        const float d = (float)(k - kmin) * du - p[2];
        const float e = expf(-0.5f * d * d * iw2);
        const float r = fmaf(p[1], e, p[0]) - yk;
        const float t = p[1] * e * d * iw2;
        const float J[4] = {1.0f, e, t, t * d * iw};
        int q = 0;
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = a; b < 4; b++) { acc[q] = fmaf(J[a], J[b], acc[q]); q++; }
#pragma unroll
        for (int a = 0; a < 4; a++) acc[10 + a] = fmaf(J[a], r, acc[10 + a]);
        acc[14] = fmaf(r, r, acc[14]);
        if constexpr (HESS) {
            float w = r * e;
#pragma unroll
            for (int j = 0; j < 5; j++) { acc[15 + j] += w; w *= d; }
        }
    };
#pragma unroll
    for (int i = 0; i < kFwCache; i++)
        if (t + kFwThreads * i < n_v) point(t + kFwThreads * i, yc[i]);
    for (int k = t + kFwThreads * kFwCache; k < n_v; k += kFwThreads) point(k, ys[k]);
    block_allsum<SPAN, NF>(acc, buf, parity);
}

template <int SPAN>
__global__ void __launch_bounds__(kFwBlock) k_gauss_fit_f32(int n_spec, int n_v_grid, double v_lo_grid,
                                                             double v_step, const double* __restrict__ ccf,
                                                             float* scratch, double* rv, double* fit,
                                                             const int* __restrict__ win) {
    constexpr int kFwThreads = Fw<SPAN>::threads, kFwCache = Fw<SPAN>::cache, kFwSpan = SPAN;
    __shared__ float buf[2 * kFwSpan * kFwMaxSums];
    __shared__ float sx[3 * kFwSpan];
    __shared__ int sk[kFwSpan];
    asm volatile("griddepcontrol.wait;" ::: "memory");      // the CCF, when launched early after it
    int parity = 0;
    const int spec = blockIdx.x * Fw<SPAN>::per_block + (int)threadIdx.x / kFwThreads;
    const int t = threadIdx.x % kFwThreads, lane = t & 31, w = t >> 5;
    if (spec >= n_spec) return;                           // SPAN = 4: the whole block; 1: the warp
    int k0 = 0, n_v = n_v_grid;
    if (win) {
        k0 = win[2 * spec];
        n_v = win[2 * spec + 1];
    }
    const double v_lo = win ? fma((double)k0, v_step, v_lo_grid) : v_lo_grid;
    const double* c = ccf + (int64_t)spec * n_v_grid + k0;
    float* ys = scratch + (int64_t)spec * n_v_grid + k0;
    // the CCF in FP32; its largest value, and its smallest with the first index reaching it
    float yc[kFwCache];
    float mx = -INFINITY, mn = INFINITY;
    int kmin = n_v;
#pragma unroll
    for (int i = 0; i < kFwCache; i++) {
        const int k = t + kFwThreads * i;
        yc[i] = k < n_v ? (float)c[k] : 0.0f;
        if (k < n_v) {
            mx = fmaxf(mx, yc[i]);
            if (yc[i] < mn) { mn = yc[i]; kmin = k; }
        }
    }
    for (int k = t + kFwThreads * kFwCache; k < n_v; k += kFwThreads) {
        const float v = (float)c[k];
        ys[k] = v;
        mx = fmaxf(mx, v);
        if (v < mn) { mn = v; kmin = k; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float mo = __shfl_xor_sync(0xffffffffu, mn, o);
        const int ko = __shfl_xor_sync(0xffffffffu, kmin, o);
        if (mo < mn || (mo == mn && ko < kmin)) { mn = mo; kmin = ko; }
    }
    if constexpr (kFwSpan > 1) {
        if (lane == 0) { sx[w] = mx; sx[kFwSpan + w] = mn; sk[w] = kmin; }
        __syncthreads();
        mx = sx[0]; mn = sx[kFwSpan]; kmin = sk[0];
#pragma unroll
        for (int v = 1; v < kFwSpan; v++) {
            mx = fmaxf(mx, sx[v]);
            const float mo = sx[kFwSpan + v];
            const int ko = sk[v];
            if (mo < mn || (mo == mn && ko < kmin)) { mn = mo; kmin = ko; }
        }
    }
    // scaled CCF y = CCF / |max|; start a = max, b = min - max, m = 0 at the minimum, w = 1 in units
    // of the starting width s0 = dip area / (|b| sqrt(2 pi)), at least one velocity step
    const float scale = mx != 0.0f ? fabsf(mx) : 1.0f;
    const float iscale = 1.0f / scale;
    float area[1] = {0.0f};
#pragma unroll
    for (int i = 0; i < kFwCache; i++) {
        yc[i] *= iscale;
        if (t + kFwThreads * i < n_v) area[0] += mx * iscale - yc[i];
    }
    for (int k = t + kFwThreads * kFwCache; k < n_v; k += kFwThreads) {   // values this thread wrote
        const float v = ys[k] * iscale;
        ys[k] = v;
        area[0] += mx * iscale - v;
    }
    block_allsum<SPAN, 1>(area, buf, parity);
    const float b0 = (mn - mx) * iscale;
    const double s0 = fmax(b0 != 0.0f ? (double)area[0] * v_step / ((double)fabsf(b0) * 2.5066282746310002) : v_step,
                           v_step);
    const double c0 = fma((double)kmin, v_step, v_lo);
    const float du = (float)(v_step / s0);

    // ---- phase 1: Levenberg-Marquardt ----
    float p[4] = {mx * iscale, b0, 0.0f, 1.0f};
    float pt[4] = {p[0], p[1], p[2], p[3]};
    float acc[15], jtj[10], jtr[4], cost = 0.0f, lam = 1e-3f;
    bool tiny = false;
    fw_pass<SPAN, false>(p, n_v, kmin, du, t, yc, ys, acc, buf, parity);
    for (int it = 0; it < kFwPassesA; it++) {
        bool stop = false;
        if (it == 0 || acc[14] <= cost) {            // keep the trial point
            for (int a = 0; a < 4; a++) p[a] = pt[a];
            for (int q = 0; q < 10; q++) jtj[q] = acc[q];
            for (int a = 0; a < 4; a++) jtr[a] = acc[10 + a];
            cost = acc[14];
            if (it > 0) lam = fmaxf(lam * 0.1f, 1e-9f);
            if (tiny) stop = true;
        } else {
            if (tiny) stop = true;
            lam *= 10.0f;
        }
        while (!stop) {
            if (lam > 1e8f) { stop = true; break; }
            float M[4][4], b[4], dx[4];
            for (int a = 0; a < 4; a++)
                for (int bb = a; bb < 4; bb++) M[a][bb] = M[bb][a] = jtj[tri(a, bb)];
            for (int a = 0; a < 4; a++) { M[a][a] *= 1.0f + lam; b[a] = -jtr[a]; }
            if (!solve4f(M, b, dx)) { lam *= 10.0f; continue; }
            tiny = fabsf(dx[2]) <= kFwTolA && fabsf(dx[3]) <= kFwTolA &&
                   fabsf(dx[0]) <= kFwTolA * fabsf(p[0]) && fabsf(dx[1]) <= kFwTolA * fabsf(p[1]);
            for (int a = 0; a < 4; a++) pt[a] = p[a] + dx[a];
            break;
        }
        if (stop) break;
        fw_pass<SPAN, false>(pt, n_v, kmin, du, t, yc, ys, acc, buf, parity);
    }

    // ---- phase 2: Newton on H = J^T J + sum r d2m ----
    float prev[4] = {p[0], p[1], p[2], p[3]};
    float cost_prev = INFINITY, last = INFINITY;
    for (int it = 0; it < kFwPassesB; it++) {
        float f[20];
        fw_pass<SPAN, true>(p, n_v, kmin, du, t, yc, ys, f, buf, parity);
        if (!(f[14] <= cost_prev * (1.0f + 1e-5f))) {   // the last step did not help: undo it
            for (int a = 0; a < 4; a++) p[a] = prev[a];
            break;
        }
        const float b = p[1], w = p[3];
        const float iw = 1.0f / w, iw2 = iw * iw;
        const float R0 = f[15], R1 = f[16], R2 = f[17], R3 = f[18], R4 = f[19];
        float M[4][4], rhs[4], dx[4];
        for (int a = 0; a < 4; a++)
            for (int bb = a; bb < 4; bb++) M[a][bb] = M[bb][a] = f[tri(a, bb)];
        M[1][2] += R1 * iw2;
        M[1][3] += R2 * iw2 * iw;
        M[2][2] += b * iw2 * (R2 * iw2 - R0);
        M[2][3] += b * iw2 * iw * (R3 * iw2 - 2.0f * R1);
        M[3][3] += b * iw2 * iw2 * (R4 * iw2 - 3.0f * R2);
        M[2][1] = M[1][2];
        M[3][1] = M[1][3];
        M[3][2] = M[2][3];
        for (int a = 0; a < 4; a++) rhs[a] = -f[10 + a];
        if (!solve4f(M, rhs, dx)) break;
        if (!(dx[0] * rhs[0] + dx[1] * rhs[1] + dx[2] * rhs[2] + dx[3] * rhs[3] > 0.0f)) break;
        const float ref = fabsf(p[0]), wref = fabsf(w);
        const float size = fmaxf(fmaxf(fabsf(dx[0]) / ref, fabsf(dx[1]) / ref),
                                 fmaxf(fabsf(dx[2]) / wref, fabsf(dx[3]) / wref));
        if (!(size < last)) break;
        for (int a = 0; a < 4; a++) { prev[a] = p[a]; p[a] += dx[a]; }
        cost_prev = f[14];
        last = size;
        if (size <= kFwTolB) break;
    }

    if (t == 0) {
        // a fit that leaves the velocity grid (no dip to fit) is reported as NaN
        const double v_hi = fma((double)(n_v - 1), v_step, v_lo);
        double mu = fma((double)p[2], s0, c0);
        if (!(mu >= v_lo && mu <= v_hi) || !(fabs((double)p[3]) * s0 <= v_hi - v_lo)) mu = NAN;
        rv[spec] = mu;
        if (fit) {
            fit[(int64_t)spec * 4 + 0] = (double)p[0] * scale;
            fit[(int64_t)spec * 4 + 1] = (double)p[1] * scale;
            fit[(int64_t)spec * 4 + 2] = mu;
            fit[(int64_t)spec * 4 + 3] = fabs((double)p[3]) * s0;
        }
    }
}

// Fits of the CCFs of FP32 spectra: a whole block per spectrum while the spectra are few (up to
// two per SM: the latency of one fit is what the call waits for), one warp per spectrum beyond
// (the throughput of many fits).
constexpr int kFwWholeBlockMax = 2 * 152;

// early: programmatic dependent launch (the kernel before it releases it; it waits for that
// kernel before it reads anything)
static cudaLaunchConfig_t pdl_config(dim3 grid, dim3 block, cudaStream_t st, bool early, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = early ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

static cudaError_t fit_f32_launch(int n_spec, cudaStream_t st, bool early, int n, int n_v, double v_lo, double v_step,
                                  const double* ccf, float* scratch, double* rv, double* fit, const int* win) {
    cudaLaunchAttribute attr[1];
    if (n_spec <= kFwWholeBlockMax) {
        const cudaLaunchConfig_t cfg = pdl_config(dim3(n_spec), dim3(kFwBlock), st, early, attr);
        return cudaLaunchKernelEx(&cfg, k_gauss_fit_f32<4>, n, n_v, v_lo, v_step, ccf, scratch, rv, fit, win);
    }
    const cudaLaunchConfig_t cfg = pdl_config(dim3((n_spec + 3) / 4), dim3(kFwBlock), st, early, attr);
    return cudaLaunchKernelEx(&cfg, k_gauss_fit_f32<1>, n, n_v, v_lo, v_step, ccf, scratch, rv, fit, win);
}

bool ccf_mask_same(const CcfState& st, const double* mask_lambda, const double* mask_weight,
                   int n_lines, double width_kms) {
    const std::vector<double>& k = st.mask_key;
    return k.size() == 2 * (size_t)n_lines + 1 &&
           std::memcmp(k.data(), mask_lambda, (size_t)n_lines * 8) == 0 &&
           std::memcmp(k.data() + n_lines, mask_weight, (size_t)n_lines * 8) == 0 &&
           std::memcmp(k.data() + 2 * (size_t)n_lines, &width_kms, 8) == 0;
}

soap_status ccf_prepare(soap_ctx* c, CcfState& st, const double* mask_lambda, const double* mask_weight,
                        int n_lines, double width_kms, double v_lo, double v_step, int n_v, int n_spec,
                        int f32, int tc, CcfPlan& p) {
    // line and velocity tables: kept while the mask, its width and the velocity grid stay the same
    const bool same_tab = st.lines_ok && st.vel_key[0] == v_lo && st.vel_key[1] == v_step &&
                          st.vel_key[2] == (double)n_v &&
                          ccf_mask_same(st, mask_lambda, mask_weight, n_lines, width_kms);
    bool sorted = true;
    if (same_tab) {
        sorted = st.sorted;
    } else {
        for (int l = 1; l < n_lines; l++)
            if (mask_lambda[l] < mask_lambda[l - 1]) { sorted = false; break; }
    }
    if ((int64_t)(n_spec + kTileSB - 1) / kTileSB > 65535) {
        set_error("%d spectra in one CCF call; at most %d", n_spec, 65535 * kTileSB);
        return SOAP_ERANGE;
    }
    p = CcfPlan{};
    p.n_spec = n_spec;
    p.n_lines = n_lines;
    p.n_v = n_v;
    p.f32 = f32;
    p.v_lo = v_lo;
    p.v_step = v_step;
    p.h = width_kms / (2.0 * kCKms * c->delta);
    // windowed kernel: one velocity per thread (n_v <= 256); blocks walk the chunks
    p.windowed = sorted && n_v <= 256 && 2.0 * width_kms / (2.0 * kCKms * c->delta) <= 15.0;
    p.n_wgroups = (n_lines + kWinLines - 1) / kWinLines;   // one chunk of lines per block
    p.n_chunks = p.windowed ? p.n_wgroups : (n_lines + kLinesPerChunk - 1) / kLinesPerChunk;
    int sms = 0, dev = 0;
    SOAP_CUDA(cudaGetDevice(&dev));
    SOAP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // register-tiled kernel (FP32, sorted mask): pixels a group of kTileVT velocities can reach
    // for one line, from the largest spread of kTileVT consecutive box positions
    if (f32 && sorted && n_v >= kTileVT) {
        const double box = width_kms / (kCKms * c->delta);
        double spread = 0.0;
        for (int k = 0; k + kTileVT - 1 < n_v; k++)
            spread = std::max(spread, (std::atanh((v_lo + (k + kTileVT - 1) * v_step) / kCKms) -
                                       std::atanh((v_lo + k * v_step) / kCKms)) / c->delta);
        const int np = (int)std::floor(spread + box + 1e-6) + 2;
        const double sweep = (std::atanh((v_lo + (n_v - 1) * v_step) / kCKms) -
                              std::atanh(v_lo / kCKms)) / c->delta + 2.0;
        const int groups = (n_v + kTileVT - 1) / kTileVT;
        if (np <= 4 && groups <= kTileMaxGroups && (groups + 15) / 16 * 16 * kTileLP <= 256 &&
            sweep + np + 5 + 1 <= kTileWin) {
            // one full wave: as many blocks as fit on the GPU at once, split evenly over the lines
            // (a partial second wave would double the time of its SMs)
            p.tile_np = std::max(np, 2);
            const int tthreads = ((groups + 15) / 16 * 16 * kTileLP + 31) / 32 * 32;
            int per_sm = 0;
            SOAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, p.tile_np == 2 ? k_ccf_tile<2, kTileSB, false>
                         : p.tile_np == 3 ? k_ccf_tile<3, kTileSB, false> : k_ccf_tile<4, kTileSB, false>,
                tthreads, 0));
            const int ys = (n_spec + kTileSB - 1) / kTileSB;
            const int wave = std::max(1, sms * std::max(per_sm, 1));
            p.tile_blocks = std::max(1, std::min(wave >= ys ? wave / ys : 1, (n_lines + 7) / 8));
            p.tile_lines = (n_lines + p.tile_blocks - 1) / p.tile_blocks;
            p.tile_blocks = (n_lines + p.tile_lines - 1) / p.tile_lines;
            p.n_chunks = p.tile_blocks;
        }
    }
    // tensor-core form (FP32 spectra, sorted mask): pixel chunks of one wave of CTAs
    if (tc && f32 && sorted && ccf_tc_fits(n_v)) {
        p.tc_chunk = ccf_tc_chunk(c->n_px, n_spec, sms);
        p.n_chunks = (int)((c->n_px + p.tc_chunk - 1) / p.tc_chunk);
        // range of the velocity shifts' integer parts S_k, one pixel of margin on each side
        double s_a = std::atanh(v_lo / kCKms) / c->delta;
        double s_b = std::atanh((v_lo + v_step * (n_v - 1)) / kCKms) / c->delta;
        p.tc_smin = (int)std::floor(std::min(s_a, s_b)) - 1;
        p.tc_smax = (int)std::floor(std::max(s_a, s_b)) + 1;
        p.tile_np = 0;
    }
    // table layout (8-byte aligned pieces, 256-byte aligned blocks) and per-call scratch
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    size_t o_lam = 0;
    size_t o_w = al(o_lam + (size_t)n_lines * 8);
    size_t o_U = al(o_w + (size_t)n_lines * 8);
    size_t o_f64 = al(o_U + (size_t)n_lines * 4);
    size_t o_f32 = al(o_f64 + (size_t)n_lines * 8);
    size_t o_w32 = al(o_f32 + (size_t)n_lines * 4);
    size_t o_valid = al(o_w32 + (size_t)n_lines * 4);
    size_t o_S = al(o_valid + (size_t)n_lines * 4);
    size_t o_g64 = al(o_S + (size_t)n_v * 4);
    size_t o_g32 = al(o_g64 + (size_t)n_v * 8);
    size_t tab_total = o_g32 + (size_t)n_v * 4;
    size_t o_part = 0;
    size_t o_ccf = al(o_part + (size_t)p.n_chunks * n_spec * n_v * 8);
    size_t o_y = al(o_ccf + (size_t)n_spec * n_v * 8);
    size_t total = o_y + (size_t)n_spec * n_v * 8;
    SOAP_TRY(ensure(st.tmp, total));
    if (!same_tab) {
        // a grown table buffer moves: the old tables (and the mask matrix) are gone with it
        st.lines_ok = false;
        st.m_ok = false;
        SOAP_TRY(ensure(st.tab, tab_total));
    }
    char* tab = st.tab.as<char>();
    char* base = st.tmp.as<char>();
    double* d_lam = (double*)(tab + o_lam);
    p.w64 = (double*)(tab + o_w);
    p.U = (int*)(tab + o_U);
    p.f64 = (double*)(tab + o_f64);
    p.f32t = (float*)(tab + o_f32);
    p.w32 = (float*)(tab + o_w32);
    p.valid = (int*)(tab + o_valid);
    p.S = (int*)(tab + o_S);
    p.g64 = (double*)(tab + o_g64);
    p.g32 = (float*)(tab + o_g32);
    p.part = (double*)(base + o_part);
    p.ccf = (double*)(base + o_ccf);
    p.y = (double*)(base + o_y);
    if (!same_tab) {
        cudaEvent_t tb = c->profiling ? timer_begin(c) : nullptr;
        const double v_hi = v_lo + v_step * (n_v - 1);
        SOAP_TRY(upload_small(c, d_lam, mask_lambda, (size_t)n_lines * 8));
        SOAP_TRY(upload_small(c, p.w64, mask_weight, (size_t)n_lines * 8));
        k_ccf_lines<<<(n_lines + 255) / 256, 256, 0, c->stream>>>(
            n_lines, d_lam, p.w64, c->lam_s, c->delta, p.h, std::atanh(v_lo / kCKms) / c->delta,
            std::atanh(v_hi / kCKms) / c->delta, c->n_px, p.U, p.f64, p.f32t, p.w32, p.valid);
        SOAP_LAUNCHED(c);
        k_ccf_velocities<<<(n_v + 127) / 128, 128, 0, c->stream>>>(n_v, v_lo, v_step, c->delta, p.S,
                                                                   p.g64, p.g32);
        SOAP_LAUNCHED(c);
        st.mask_key.assign(mask_lambda, mask_lambda + n_lines);
        st.mask_key.insert(st.mask_key.end(), mask_weight, mask_weight + n_lines);
        st.mask_key.push_back(width_kms);
        st.vel_key[0] = v_lo;
        st.vel_key[1] = v_step;
        st.vel_key[2] = (double)n_v;
        st.sorted = sorted;
        st.lines_ok = true;
        if (tb) timer_end(c, SOAP_TIMER_CCF_AUX, tb);
    }
    if (p.tc_chunk && !st.m_ok) SOAP_TRY(ccf_tc_build_m(c, st, p));
    return SOAP_OK;
}

soap_status ccf_enqueue(soap_ctx* c, CcfState& st, const CcfPlan& p, const void* spectra_dev, double* rv_dev,
                        double* fit_dev, double* ccf_dev, const int* win) {
    const int n_spec = p.n_spec, n_v = p.n_v, n_lines = p.n_lines;
    double* d_part = p.part;
    double* d_ccf = ccf_dev ? ccf_dev : p.ccf;
    cudaEvent_t tb = c->profiling ? timer_begin(c) : nullptr;
    const int threads = n_v >= 256 ? 256 : ((n_v + 31) / 32) * 32;
    if (p.tc_chunk) {
        SOAP_TRY(ccf_tc(c, st, p, (const float*)spectra_dev, reinterpret_cast<float*>(d_part)));
    } else if (p.tile_np) {
        const int tthreads = (((n_v + kTileVT - 1) / kTileVT + 15) / 16 * 16 * kTileLP + 31) / 32 * 32;
        const float box = (float)(2.0 * p.h);
        const bool skip0 = 2.0 * p.h <= 1.0;             // boxes no wider than a pixel
        const int n16 = (n_spec + kTileSB - 1) / kTileSB;   // blocks of 16 spectra (the last ragged)
#define SOAP_TILE_LAUNCH(NP, SB, SK, NB, SBASE)                                                    \
        k_ccf_tile<NP, SB, SK><<<dim3((unsigned)p.tile_blocks, (unsigned)(NB)), tthreads, 0, c->stream>>>( \
            n_lines, p.tile_lines, p.U, p.f32t, p.valid, p.w32, n_v, p.S, p.g32, box, c->n_px, n_spec,   \
            SBASE, (const float*)spectra_dev, reinterpret_cast<float*>(d_part))
#define SOAP_TILE_NP(SB, NB, SBASE)                                                                \
        do {                                                                                       \
            if (p.tile_np == 2) SOAP_TILE_LAUNCH(2, SB, false, NB, SBASE);                         \
            else if (p.tile_np == 3 && skip0) SOAP_TILE_LAUNCH(3, SB, true, NB, SBASE);            \
            else if (p.tile_np == 3) SOAP_TILE_LAUNCH(3, SB, false, NB, SBASE);                    \
            else if (skip0) SOAP_TILE_LAUNCH(4, SB, true, NB, SBASE);                              \
            else SOAP_TILE_LAUNCH(4, SB, false, NB, SBASE);                                        \
        } while (0)
        SOAP_TILE_NP(kTileSB, n16, 0);
#undef SOAP_TILE_NP
#undef SOAP_TILE_LAUNCH
    } else if (p.windowed) {
        const int threads = ((n_v + 31) / 32) * 32;
        const double box = 2.0 * p.h;
        const bool small = box <= 1.0;                   // the box covers at most 2 pixels
        dim3 grid32((unsigned)p.n_wgroups, (unsigned)((n_spec + 15) / 16));
        dim3 grid64((unsigned)p.n_wgroups, (unsigned)((n_spec + 7) / 8));
        const size_t smem32 = (size_t)kWinMax * (16 + 4) * 4;
        const size_t smem64 = (size_t)kWinMax * (8 + 2) * 8;
#define SOAP_CCF_LAUNCH(T, SB, NB, GRID, SMEM, F, WT, G, SPEC)                                    \
        do {                                                                                       \
            SOAP_CUDA(cudaFuncSetAttribute(k_ccf_window<T, SB, NB>,                                \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM)); \
            k_ccf_window<T, SB, NB><<<GRID, threads, SMEM, c->stream>>>(                          \
                n_lines, p.U, F, p.valid, WT, n_v, p.S, G, box, c->n_px, n_spec,                   \
                (const T*)SPEC, reinterpret_cast<T*>(d_part));                                     \
        } while (0)
        if (p.f32) {
            if (small) SOAP_CCF_LAUNCH(float, 16, 2, grid32, smem32, p.f32t, p.w32, p.g32, spectra_dev);
            else SOAP_CCF_LAUNCH(float, 16, 16, grid32, smem32, p.f32t, p.w32, p.g32, spectra_dev);
        } else {
            if (small) SOAP_CCF_LAUNCH(double, 8, 2, grid64, smem64, p.f64, p.w64, p.g64, spectra_dev);
            else SOAP_CCF_LAUNCH(double, 8, 16, grid64, smem64, p.f64, p.w64, p.g64, spectra_dev);
        }
#undef SOAP_CCF_LAUNCH
    } else if (p.f32) {
        constexpr int SB = 16;
        dim3 grid((unsigned)p.n_chunks, (unsigned)((n_spec + SB - 1) / SB));
        k_ccf_partial<float, SB><<<grid, threads, 0, c->stream>>>(
            n_lines, p.U, p.f32t, p.valid, p.w64, n_v, p.S, p.g32, 2.0 * p.h, c->n_px, n_spec,
            (const float*)spectra_dev, d_part);
    } else {
        constexpr int SB = 8;
        dim3 grid((unsigned)p.n_chunks, (unsigned)((n_spec + SB - 1) / SB));
        k_ccf_partial<double, SB><<<grid, threads, 0, c->stream>>>(
            n_lines, p.U, p.f64, p.valid, p.w64, n_v, p.S, p.g64, 2.0 * p.h, c->n_px, n_spec,
            (const double*)spectra_dev, d_part);
    }
    SOAP_LAUNCHED(c);
    if (tb) timer_end(c, SOAP_TIMER_CCF, tb);
    tb = c->profiling ? timer_begin(c) : nullptr;
    const unsigned rblocks = (unsigned)(((int64_t)n_spec * n_v + 31) / 32);
    // after the tensor-core CCF (which releases its dependents as it starts) the reduction and the
    // fit are launched early, so that their launches overlap the kernel before them
    const bool early = p.tc_chunk != 0;
    if ((p.windowed || p.tile_np || p.tc_chunk) && p.f32) {  // FP32 partial sums (converted exactly to FP64 here)
        cudaLaunchAttribute attr[1];
        const cudaLaunchConfig_t cfg = pdl_config(dim3(rblocks), dim3(32, kReduceSplit), c->stream, early, attr);
        SOAP_CUDA(cudaLaunchKernelEx(&cfg, k_ccf_reduce<float>, p.n_chunks, n_spec, n_v,
                                     reinterpret_cast<const float*>(d_part), d_ccf));
    } else
        k_ccf_reduce<double><<<rblocks, dim3(32, kReduceSplit), 0, c->stream>>>(p.n_chunks, n_spec, n_v,
                                                                                d_part, d_ccf);
    SOAP_LAUNCHED(c);
    if (tb) timer_end(c, SOAP_TIMER_CCF_AUX, tb);
    if (p.f32)      // float32 spectra: FP32 fit, one warp per spectrum
        SOAP_TIMED(c, SOAP_TIMER_FIT,
                   SOAP_CUDA(fit_f32_launch(n_spec, c->stream, early,
                       n_spec, n_v, p.v_lo, p.v_step, d_ccf, reinterpret_cast<float*>(p.y), rv_dev, fit_dev, win));
                   SOAP_LAUNCHED(c));
    else            // float64 spectra: FP64 residuals, the least-squares minimum to FP64 rounding
        SOAP_TIMED(c, SOAP_TIMER_FIT,
                   k_gauss_fit<<<n_spec, kFitThreads, 0, c->stream>>>(n_spec, n_v, p.v_lo, p.v_step, d_ccf, p.y,
                                                                      rv_dev, fit_dev, win);
                   SOAP_LAUNCHED(c));
    return SOAP_OK;
}

soap_status rv_ccf_run(soap_ctx* c, const void* spectra_dev, int f32, int n_spec,
                       const double* mask_lambda, const double* mask_weight, int n_lines,
                       double width_kms, double v_lo, double v_step, int n_v, double* rv_dev,
                       double* fit_dev, double* ccf_dev, int tc) {
    CcfPlan p;
    SOAP_TRY(ccf_prepare(c, c->ccf, mask_lambda, mask_weight, n_lines, width_kms, v_lo, v_step, n_v, n_spec,
                         f32, tc, p));
    return ccf_enqueue(c, c->ccf, p, spectra_dev, rv_dev, fit_dev, ccf_dev, nullptr);
}

}  // namespace soap

// ---------------------------------------------------------------------------------------
// Allocation-free variant of the CCF + RV fit (soap_rv_ccf_static in soap.h)
// ---------------------------------------------------------------------------------------
// Some callers may not allocate device memory once they are running: applications that
// hand every byte of the GPU to their own pool at start-up, real-time pipelines where an
// allocation (which can synchronise the device) is not allowed after initialisation, or
// plug-ins that only receive buffers from their host.  For them this entry point works on
// caller buffers only; its scratch is the fixed array below, which every GPU that loads the
// library holds until the process exits.
namespace soap {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;      // 16 MiB
static __device__ __align__(256) unsigned char g_rv_scratch[kStaticScratchBytes];

constexpr int kStaticMaxDevices = 64;
static std::atomic<void*> g_rv_scratch_ptr[kStaticMaxDevices];   // device address per device
static std::mutex g_rv_scratch_mutex;                            // serialises first lookups

// Device address of g_rv_scratch on the current device, looked up once per device.  In host
// code g_rv_scratch is only a host-side handle, so the address must come from the runtime.
// Threads making their first call at the same time take the lookup in turn; later calls read
// the cached address without locking.
static soap_status static_scratch(void** out) {
    int dev = 0;
    SOAP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kStaticMaxDevices) {
        set_error("device %d beyond the %d devices soap_rv_ccf_static supports", dev, kStaticMaxDevices);
        return SOAP_ERANGE;
    }
    void* p = g_rv_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(g_rv_scratch_mutex);
        p = g_rv_scratch_ptr[dev].load(std::memory_order_acquire);
        if (!p) {
            cudaError_t e = cudaGetSymbolAddress(&p, g_rv_scratch);
            if (e != cudaSuccess || !p) {
                set_error("cudaGetSymbolAddress(g_rv_scratch) failed: %s", cudaGetErrorString(e));
                return SOAP_ECUDA;
            }
            g_rv_scratch_ptr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return SOAP_OK;
}

}  // namespace soap

extern "C" soap_status soap_rv_ccf_static(double lambda_start_A, double lambda_end_A, int64_t n_px,
                                          const void* spectra, int32_t spectra_f32, int32_t n_spec,
                                          const double* mask_lambda, const double* mask_weight,
                                          int32_t n_lines, double mask_width_kms, double v_lo,
                                          double v_step, int32_t n_v, double* rv_kms,
                                          double* fit_params, double* ccf_out, void* cuda_stream) {
    using namespace soap;
    clear_error();
    if (!spectra || !mask_lambda || !mask_weight || !rv_kms) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (spectra_f32 != 0 && spectra_f32 != 1) { set_error("spectra_f32 must be 0 or 1"); return SOAP_EINVAL; }
    if (!(lambda_start_A > 0) || !(lambda_end_A > lambda_start_A) || !std::isfinite(lambda_end_A) ||
        n_px < 2 || n_px > (int64_t(1) << 28)) {
        set_error("invalid wavelength grid"); return SOAP_EINVAL;
    }
    if (n_spec < 0 || n_lines < 1 || n_v < 5 || n_v > 4096) { set_error("need n_spec >= 0, n_lines >= 1, 5 <= n_v <= 4096"); return SOAP_EINVAL; }
    if (!std::isfinite(mask_width_kms) || !(mask_width_kms > 0) || !std::isfinite(v_lo) ||
        !std::isfinite(v_step) || !(v_step > 0)) {
        set_error("mask width / velocity grid invalid"); return SOAP_EINVAL;
    }
    const double v_hi = v_lo + v_step * (n_v - 1);
    if (!(std::fabs(v_lo) < kCKms) || !(std::fabs(v_hi) < kCKms)) { set_error("velocity grid reaches c"); return SOAP_EINVAL; }
    const double delta = std::log1p((lambda_end_A - lambda_start_A) / lambda_start_A) / (double)(n_px - 1);
    const double h = mask_width_kms / (2.0 * kCKms * delta);
    if (2.0 * h > 14.0) { set_error("mask box spans more than 14 pixels"); return SOAP_ERANGE; }
    if (n_spec == 0) return SOAP_OK;
    // scratch layout, as in rv_ccf_run (generic line order kernel)
    const int n_chunks = (n_lines + kLinesPerChunk - 1) / kLinesPerChunk;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    size_t o_U = 0;
    size_t o_f64 = al(o_U + (size_t)n_lines * 4);
    size_t o_f32 = al(o_f64 + (size_t)n_lines * 8);
    size_t o_w32 = al(o_f32 + (size_t)n_lines * 4);
    size_t o_valid = al(o_w32 + (size_t)n_lines * 4);
    size_t o_S = al(o_valid + (size_t)n_lines * 4);
    size_t o_g64 = al(o_S + (size_t)n_v * 4);
    size_t o_g32 = al(o_g64 + (size_t)n_v * 8);
    size_t o_part = al(o_g32 + (size_t)n_v * 4);
    size_t o_ccf = al(o_part + (size_t)n_chunks * n_spec * n_v * 8);
    size_t o_y = al(o_ccf + (size_t)n_spec * n_v * 8);
    size_t total = o_y + (size_t)n_spec * n_v * 8;
    if (total > kStaticScratchBytes) {
        set_error("soap_rv_ccf_static needs %zu bytes of scratch for %d lines x %d spectra x %d velocities; "
                  "its fixed scratch holds %zu (use fewer spectra per call, or soap_rv_ccf)",
                  total, n_lines, n_spec, n_v, kStaticScratchBytes);
        return SOAP_ERANGE;
    }
    void* sp = nullptr;
    SOAP_TRY(static_scratch(&sp));
    char* base = static_cast<char*>(sp);
    int* d_U = (int*)(base + o_U);
    double* d_f64 = (double*)(base + o_f64);
    float* d_f32 = (float*)(base + o_f32);
    float* d_w32 = (float*)(base + o_w32);
    int* d_valid = (int*)(base + o_valid);
    int* d_S = (int*)(base + o_S);
    double* d_g64 = (double*)(base + o_g64);
    float* d_g32 = (float*)(base + o_g32);
    double* d_part = (double*)(base + o_part);
    double* d_ccf = ccf_out ? ccf_out : (double*)(base + o_ccf);
    double* d_y = (double*)(base + o_y);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    // every scratch element read below is written earlier in this call: nothing needs clearing
    k_ccf_lines<<<(n_lines + 255) / 256, 256, 0, stream>>>(
        n_lines, mask_lambda, mask_weight, lambda_start_A, delta, h, std::atanh(v_lo / kCKms) / delta,
        std::atanh(v_hi / kCKms) / delta, n_px, d_U, d_f64, d_f32, d_w32, d_valid);
    SOAP_CUDA(cudaGetLastError());
    k_ccf_velocities<<<(n_v + 127) / 128, 128, 0, stream>>>(n_v, v_lo, v_step, delta, d_S, d_g64, d_g32);
    SOAP_CUDA(cudaGetLastError());
    const int threads = n_v >= 256 ? 256 : ((n_v + 31) / 32) * 32;
    if (spectra_f32) {
        constexpr int SB = 16;
        dim3 grid((unsigned)n_chunks, (unsigned)((n_spec + SB - 1) / SB));
        k_ccf_partial<float, SB><<<grid, threads, 0, stream>>>(
            n_lines, d_U, d_f32, d_valid, mask_weight, n_v, d_S, d_g32, 2.0 * h, n_px, n_spec,
            (const float*)spectra, d_part);
    } else {
        constexpr int SB = 8;
        dim3 grid((unsigned)n_chunks, (unsigned)((n_spec + SB - 1) / SB));
        k_ccf_partial<double, SB><<<grid, threads, 0, stream>>>(
            n_lines, d_U, d_f64, d_valid, mask_weight, n_v, d_S, d_g64, 2.0 * h, n_px, n_spec,
            (const double*)spectra, d_part);
    }
    SOAP_CUDA(cudaGetLastError());
    k_ccf_reduce<double><<<(unsigned)(((int64_t)n_spec * n_v + 31) / 32), dim3(32, kReduceSplit), 0, stream>>>(
        n_chunks, n_spec, n_v, d_part, d_ccf);
    SOAP_CUDA(cudaGetLastError());
    if (spectra_f32)
        SOAP_CUDA(fit_f32_launch(n_spec, stream, false,
            n_spec, n_v, v_lo, v_step, d_ccf, reinterpret_cast<float*>(d_y), rv_kms, fit_params, nullptr));
    else
        k_gauss_fit<<<n_spec, kFitThreads, 0, stream>>>(n_spec, n_v, v_lo, v_step, d_ccf, d_y, rv_kms, fit_params,
                                                        nullptr);
    SOAP_CUDA(cudaGetLastError());
    return SOAP_OK;
}
