// contract_dev.cuh -- device code of the Toeplitz contraction shared by the single-star
// kernels (contract.cu) and the batched persistent kernel (batch.cu).
//
// contract_tile() computes one pixel tile of one block of PB phases:
//   out[p][m] = F_q[m] - sum_b Q_p,b * S_q,b [m] + sum_cl C_cl[m] sum_b K_p,cl,b * S_a(cl),b [m]
// (Eqs. 1-4 for the effect `eff`), from a tap table (group starts, per-tap row offsets,
// coefficients [tap][PB]).  One thread owns R pixels m = m0 + threadIdx.x + r*THREADS; acc
// holds F_q - group 0 + folded class terms, tmp one class before its fold.
#pragma once

#include "soap_internal.cuh"

namespace soap {

template <typename T>
struct Rows {
    const T* q;         // quiet rows [n_mu][row_len]
    const T* a[2];      // active rows spot / facula
};

struct ClassTypes {
    int t[SOAP_MAX_CLASSES];
};

struct EffectList {
    int e[3];
};

// PB coefficients of one tap (16-byte vector loads when PB allows; coefficient slabs are
// 256-byte aligned and every job's block is a multiple of PB elements).
template <typename T, int PB>
__device__ __forceinline__ void load_coefs(const T* __restrict__ src, T (&cv)[PB]) {
    if constexpr (sizeof(T) == 4 && PB % 4 == 0) {
#pragma unroll
        for (int q = 0; q < PB / 4; q++) {
            const float4 t = __ldg(reinterpret_cast<const float4*>(src) + q);
            cv[4 * q] = t.x; cv[4 * q + 1] = t.y; cv[4 * q + 2] = t.z; cv[4 * q + 3] = t.w;
        }
    } else if constexpr (sizeof(T) == 8 && PB % 2 == 0) {
#pragma unroll
        for (int q = 0; q < PB / 2; q++) {
            const double2 t = __ldg(reinterpret_cast<const double2*>(src) + q);
            cv[2 * q] = t.x; cv[2 * q + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int p = 0; p < PB; p++) cv[p] = __ldg(src + p);
    }
}

// Region classes as the contraction sees them: the type of class cl (which active rows it
// convolves) and its contrast C_cl at pixel m.  TableContrast reads precomputed rows
// [n_class][n_px]; PlanckContrast32 evaluates the Planck ratio of Sect. 4.3.1 in FP32 with the
// same operations as k_contrast32 (so both give the same values).
template <typename T>
struct TableContrast {
    const T* rows;
    int64_t n_px;
    ClassTypes ct;
    __device__ __forceinline__ int type(int cl) const { return ct.t[cl]; }
    __device__ __forceinline__ T at(int cl, int64_t m) const { return rows[(int64_t)cl * n_px + m]; }
};

struct PlanckContrast32 {
    float aq, fd;            // h c / (lambda_s k T_quiet), grid step Delta
    const int* types;        // [n_class]
    const float* a;          // [n_class]: h c / (lambda_s k T_class)
    __device__ __forceinline__ int type(int cl) const { return types[cl]; }
    __device__ __forceinline__ float at(int cl, int64_t m) const {
        const float inv = expf(-(float)m * fd);            // lambda_s / lambda_m
        return expm1f(aq * inv) / expm1f(a[cl] * inv);
    }
};

// bs (optional): per-(group, mu bin) tap starts [G n_mu + 1]; with it each class is folded
// per bin, acc += C_(cl n_mu + b)[m] . sum_(taps of bin b) (a contrast row per class and bin:
// mu-dependent facula temperatures).
template <typename T, int PB, int R, int THREADS, class Con>
__device__ __forceinline__ void contract_tile(int64_t n_px, const Rows<T>& rows, const long long* __restrict__ toff,
                                              const int* __restrict__ gs, int G, const T* __restrict__ cb,
                                              const Con& con, const T* __restrict__ fq, int eff, int64_t tile,
                                              int np, T* __restrict__ out_rows, const int* __restrict__ bs = nullptr,
                                              int n_mu = 0) {
    // Rows are padded past round_up(n_px, 1024) + max tap, so every tap of every pixel of the
    // last tile reads inside its row; only the per-pixel inputs below need a clamped index.
    const int64_t m0 = tile * THREADS * R + threadIdx.x;
    int64_t mcl[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int64_t m = m0 + (int64_t)r * THREADS;
        mcl[r] = m < n_px ? m : n_px - 1;
    }
    // The tap sums accumulate from zero and F_q is added once at the store: every FMA then
    // rounds at the scale of the residual, not of the continuum (about 8x finer in FP32).
    T acc[PB][R];
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
        for (int p = 0; p < PB; p++) acc[p][r] = T(0);
    // group 0: subtract (active star) or add (quiet star) the quiet-row convolutions
    {
        const T* base = rows.q + m0;
        const int t1 = gs[1];
#pragma unroll 4
        for (int t = gs[0]; t < t1; t++) {
            const T* row = base + __ldg(toff + t);
            T s[R];
#pragma unroll
            for (int r = 0; r < R; r++) s[r] = __ldg(row + r * THREADS);
            T cv[PB];
            load_coefs<T, PB>(cb + (int64_t)t * PB, cv);
#pragma unroll
            for (int p = 0; p < PB; p++)
#pragma unroll
                for (int r = 0; r < R; r++) acc[p][r] = fma(cv[p], s[r], acc[p][r]);
        }
    }
    // classes with a contrast row per mu bin: fold each bin's sum separately
    if (bs) {
        for (int g = 1; g < G; g++) {
            if (gs[g] == gs[g + 1]) continue;
            const int cl = g - 1;
            const T* base = (eff == SOAP_EFFECT_FLUX ? rows.q : rows.a[con.type(cl) == SOAP_FACULA ? 1 : 0]) + m0;
            for (int b = 0; b < n_mu; b++) {
                const int t0 = bs[g * n_mu + b], t1 = bs[g * n_mu + b + 1];
                if (t0 == t1) continue;
                T tmp[PB][R];
#pragma unroll
                for (int p = 0; p < PB; p++)
#pragma unroll
                    for (int r = 0; r < R; r++) tmp[p][r] = T(0);
                for (int t = t0; t < t1; t++) {
                    const T* row = base + __ldg(toff + t);
                    T s[R];
#pragma unroll
                    for (int r = 0; r < R; r++) s[r] = __ldg(row + r * THREADS);
                    T cv[PB];
                    load_coefs<T, PB>(cb + (int64_t)t * PB, cv);
#pragma unroll
                    for (int p = 0; p < PB; p++)
#pragma unroll
                        for (int r = 0; r < R; r++) tmp[p][r] = fma(cv[p], s[r], tmp[p][r]);
                }
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const T cr = eff == SOAP_EFFECT_BCONV ? T(1) : con.at(cl * n_mu + b, mcl[r]);
#pragma unroll
                    for (int p = 0; p < PB; p++) acc[p][r] = fma(cr, tmp[p][r], acc[p][r]);
                }
            }
        }
        G = 1;                                             // classes done
    }
    // classes: tmp = sum_b K_cl,b * S, then acc += C_cl . tmp (TOT, FLUX) or tmp (BCONV)
    for (int g = 1; g < G; g++) {
        const int t0 = gs[g], t1 = gs[g + 1];
        if (t0 == t1) continue;
        const int cl = g - 1;
        const T* base = (eff == SOAP_EFFECT_FLUX ? rows.q : rows.a[con.type(cl) == SOAP_FACULA ? 1 : 0]) + m0;
        T tmp[PB][R];
#pragma unroll
        for (int p = 0; p < PB; p++)
#pragma unroll
            for (int r = 0; r < R; r++) tmp[p][r] = T(0);
#pragma unroll 4
        for (int t = t0; t < t1; t++) {
            const T* row = base + __ldg(toff + t);
            T s[R];
#pragma unroll
            for (int r = 0; r < R; r++) s[r] = __ldg(row + r * THREADS);
            T cv[PB];
            load_coefs<T, PB>(cb + (int64_t)t * PB, cv);
#pragma unroll
            for (int p = 0; p < PB; p++)
#pragma unroll
                for (int r = 0; r < R; r++) tmp[p][r] = fma(cv[p], s[r], tmp[p][r]);
        }
#pragma unroll
        for (int r = 0; r < R; r++) {
            const T cr = eff == SOAP_EFFECT_BCONV ? T(1) : con.at(cl, mcl[r]);
#pragma unroll
            for (int p = 0; p < PB; p++) acc[p][r] = fma(cr, tmp[p][r], acc[p][r]);
        }
    }
    // store out_rows[p][m]
#pragma unroll
    for (int p = 0; p < PB; p++) {
        if (p >= np) break;
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int64_t m = m0 + (int64_t)r * THREADS;
            if (m < n_px) out_rows[(int64_t)p * n_px + m] = fq ? fq[mcl[r]] + acc[p][r] : acc[p][r];
        }
    }
}


// Folded form for tap tables without the quiet group (builder mode 2: group g = class g): the
// quiet rows enter each class's operand, X_cl[m - k] = Ca_cl[m] S_a(cl)[m - k] + Cq_cl[m] S_q[m - k]
// with (Ca, Cq) = (C_cl, -1) for the total effect, (0, C_cl - 1) for the flux effect and (1, -1)
// for the convective blueshift effect, so that out[p][m] = F_q[m] + sum_cl sum_taps K X (the
// quiet group's kernel is -sum_cl K_cl): one coefficient vector and one FMA per phase and pixel
// per tap instead of two.  Classes with a contrast row per mu bin keep contract_tile.
template <typename T, int PB, int R, int THREADS, class Con>
__device__ __forceinline__ void contract_tile_fold(int64_t n_px, const Rows<T>& rows,
                                                   const long long* __restrict__ toff, const int* __restrict__ gs,
                                                   int G, const T* __restrict__ cb, const Con& con,
                                                   const T* __restrict__ fq, int eff, int64_t tile, int np,
                                                   T* __restrict__ out_rows) {
    const int64_t m0 = tile * THREADS * R + threadIdx.x;
    int64_t mcl[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int64_t m = m0 + (int64_t)r * THREADS;
        mcl[r] = m < n_px ? m : n_px - 1;
    }
    T acc[PB][R];
#pragma unroll
    for (int p = 0; p < PB; p++)
#pragma unroll
        for (int r = 0; r < R; r++) acc[p][r] = T(0);
    const T* bq = rows.q + m0;
    for (int g = 0; g < G; g++) {
        const int t0 = gs[g], t1 = gs[g + 1];
        if (t0 == t1) continue;
        const T* ba = (eff == SOAP_EFFECT_FLUX ? rows.q : rows.a[con.type(g) == SOAP_FACULA ? 1 : 0]) + m0;
        T ca[R], cq[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const T C = eff == SOAP_EFFECT_BCONV ? T(1) : con.at(g, mcl[r]);
            ca[r] = eff == SOAP_EFFECT_FLUX ? T(0) : C;
            cq[r] = eff == SOAP_EFFECT_FLUX ? C - T(1) : T(-1);
        }
#pragma unroll 4
        for (int t = t0; t < t1; t++) {
            const long long off = __ldg(toff + t);
            T x[R];
#pragma unroll
            for (int r = 0; r < R; r++)
                x[r] = fma(ca[r], __ldg(ba + off + r * THREADS), cq[r] * __ldg(bq + off + r * THREADS));
            T cv[PB];
            load_coefs<T, PB>(cb + (int64_t)t * PB, cv);
#pragma unroll
            for (int p = 0; p < PB; p++)
#pragma unroll
                for (int r = 0; r < R; r++) acc[p][r] = fma(cv[p], x[r], acc[p][r]);
        }
    }
#pragma unroll
    for (int p = 0; p < PB; p++) {
        if (p >= np) break;
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int64_t m = m0 + (int64_t)r * THREADS;
            if (m < n_px) out_rows[(int64_t)p * n_px + m] = fq ? fq[mcl[r]] + acc[p][r] : acc[p][r];
        }
    }
}

// FP32 form of contract_tile_fold with the effect fixed at compile time: X = C S_a - S_q (TOT),
// S_a - S_q (BCONV), (C - 1) S_q (FLUX, no active row read), the same roundings as the generic
// form, and the accumulators of pixel pairs (r, r+1) in 64-bit registers updated by two-wide
// FMAs (fma.rn.f32x2: two independent IEEE FMAs), so the results are the same.
__device__ __forceinline__ unsigned long long ct_pack(float lo, float hi) {
    unsigned long long v;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(lo), "f"(hi));
    return v;
}
__device__ __forceinline__ void ct_unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ void ct_fma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

template <int PB, int R, int THREADS, int EFF, class Con>
__device__ __forceinline__ void contract_tile_fold32(int64_t n_px, const Rows<float>& rows,
                                                     const long long* __restrict__ toff,
                                                     const int* __restrict__ gs, int G, const float* __restrict__ cb,
                                                     const Con& con, const float* __restrict__ fq, int64_t tile,
                                                     int np, float* __restrict__ out_rows) {
    static_assert(R % 2 == 0, "pixel pairs");
    const int64_t m0 = tile * THREADS * R + threadIdx.x;
    int64_t mcl[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int64_t m = m0 + (int64_t)r * THREADS;
        mcl[r] = m < n_px ? m : n_px - 1;
    }
    unsigned long long acc[PB][R / 2];
#pragma unroll
    for (int p = 0; p < PB; p++)
#pragma unroll
        for (int k = 0; k < R / 2; k++) acc[p][k] = 0ull;
    const float* bq = rows.q + m0;
    for (int g = 0; g < G; g++) {
        const int t0 = gs[g], t1 = gs[g + 1];
        if (t0 == t1) continue;
        const float* ba = rows.a[con.type(g) == SOAP_FACULA ? 1 : 0] + m0;
        float cc[R];                                       // C (TOT) or C - 1 (FLUX)
#pragma unroll
        for (int r = 0; r < R; r++) {
            if constexpr (EFF == SOAP_EFFECT_BCONV) cc[r] = 1.0f;
            else if constexpr (EFF == SOAP_EFFECT_FLUX) cc[r] = con.at(g, mcl[r]) - 1.0f;
            else cc[r] = con.at(g, mcl[r]);
        }
#pragma unroll 4
        for (int t = t0; t < t1; t++) {
            const long long off = __ldg(toff + t);
            float x[R];
#pragma unroll
            for (int r = 0; r < R; r++) {
                const float q = __ldg(bq + off + r * THREADS);
                if constexpr (EFF == SOAP_EFFECT_FLUX) x[r] = cc[r] * q;
                else if constexpr (EFF == SOAP_EFFECT_BCONV) x[r] = __ldg(ba + off + r * THREADS) - q;
                else x[r] = fmaf(cc[r], __ldg(ba + off + r * THREADS), -q);
            }
            unsigned long long x2[R / 2];
#pragma unroll
            for (int k = 0; k < R / 2; k++) x2[k] = ct_pack(x[2 * k], x[2 * k + 1]);
            float cv[PB];
            load_coefs<float, PB>(cb + (int64_t)t * PB, cv);
#pragma unroll
            for (int p = 0; p < PB; p++) {
                const unsigned long long c2 = ct_pack(cv[p], cv[p]);
#pragma unroll
                for (int k = 0; k < R / 2; k++) ct_fma2(acc[p][k], c2, x2[k]);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < PB; p++) {
        if (p >= np) break;
        float y[R];
#pragma unroll
        for (int k = 0; k < R / 2; k++) ct_unpack(acc[p][k], y[2 * k], y[2 * k + 1]);
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int64_t m = m0 + (int64_t)r * THREADS;
            if (m < n_px) out_rows[(int64_t)p * n_px + m] = fq ? fq[mcl[r]] + y[r] : y[r];
        }
    }
}

// Contrast rows from a device list of temperatures (one row per class and mu bin when facula
// temperatures depend on mu): FP64 rows (and their FP32 copies).
static __global__ void k_contrast_rows(int64_t n_px, double lam_s, double delta, double t_quiet, int n_rows,
                                       const double* __restrict__ temps, double* c64, float* c32) {
    const double hck = kPlanckH * kLightSI / kBoltzmann * 1e10;   // Angstrom Kelvin
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n_px;
         m += (int64_t)gridDim.x * blockDim.x) {
        const double lam = lam_s * exp((double)m * delta);
        const double xq = expm1(hck / (lam * t_quiet));
        for (int k = blockIdx.y; k < n_rows; k += gridDim.y) {
            const double v = xq / expm1(hck / (lam * temps[k]));
            c64[(int64_t)k * n_px + m] = v;
            c32[(int64_t)k * n_px + m] = (float)v;
        }
    }
}

// FP32 rows with the operations of k_contrast32 (a = h c / (lambda_s k T) per row).
static __global__ void k_contrast_rows32(int64_t n_px, float aq, float fd, int n_rows, const float* __restrict__ a,
                                         float* c32) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n_px;
         m += (int64_t)gridDim.x * blockDim.x) {
        const float inv = expf(-(float)m * fd);            // lambda_s / lambda_m
        const float xq = expm1f(aq * inv);
        for (int k = blockIdx.y; k < n_rows; k += gridDim.y)
            c32[(int64_t)k * n_px + m] = xq / expm1f(a[k] * inv);
    }
}

// FP32 contrast per class (relative error ~1e-7, inside the mixed path's 2e-6).
struct ClassConsts {
    float a[SOAP_MAX_CLASSES];       // h c / (lambda_s k T_class)
};

static __global__ void k_contrast32(int64_t n_px, float aq, float fd, int n_class, ClassConsts ac, float* c32) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n_px;
         m += (int64_t)gridDim.x * blockDim.x) {
        const float inv = expf(-(float)m * fd);            // lambda_s / lambda_m
        const float xq = expm1f(aq * inv);
        for (int cl = 0; cl < n_class; cl++) c32[cl * n_px + m] = xq / expm1f(ac.a[cl] * inv);
    }
}

// ---------------------------------------------------------------------------------------
// regions (Alg. 5): centre, cap and cell box per (phase, region), and the InfoMap owner
// ---------------------------------------------------------------------------------------
struct RegionGeo {
    double P[3];       // unit vector of the cap centre, observer frame
    double cosr;       // cos of the cap's angular radius, sqrt(1 - r^2)
    float Pf[3];
    float cosrf;
    int box[4];        // i0, i1, j0, j1 (empty if i1 < i0)
    int cls;
    int pad;
};

// Region centre at `phase` (observer frame, rotation axis (0, sin i, cos i)): star-frame
// (cos lat sin L, sin lat, cos lat cos L) with L = lon + 360 phase (1 + alpha sin^2 lat), tilted
// by the inclination; written with explicitly rounded FP64 steps.  The cell box is
// conservative: the cap reaches axis angles within +-asin(r) of the centre's.
__device__ __forceinline__ RegionGeo region_geometry(int N, const RegionDev& g, double phase, double incl_deg,
                                                     double alpha) {
    const double d2r = kPi / 180.0;
    const double lat = __dmul_rn(g.lat_deg, d2r);
    double sl, cl;
    sincos(lat, &sl, &cl);
    const double lonp = __dadd_rn(g.lon_deg, __dmul_rn(__dmul_rn(360.0, phase),
                                                       __dadd_rn(1.0, __dmul_rn(__dmul_rn(alpha, sl), sl))));
    const double lon = __dmul_rn(lonp, d2r);
    const double incl = __dmul_rn(incl_deg, d2r);
    double si, ci, sn, cn;
    sincos(incl, &si, &ci);
    sincos(lon, &sn, &cn);
    const double px = __dmul_rn(cl, sn), py = sl, pz = __dmul_rn(cl, cn);
    RegionGeo o;
    o.P[0] = px;
    o.P[1] = __dsub_rn(__dmul_rn(py, si), __dmul_rn(pz, ci));
    o.P[2] = __dadd_rn(__dmul_rn(py, ci), __dmul_rn(pz, si));
    const double r = g.radius;
    o.cosr = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(r, r)));
    for (int k = 0; k < 3; k++) o.Pf[k] = (float)o.P[k];
    o.cosrf = (float)o.cosr;
    o.cls = g.cls;
    o.pad = 0;
    // The cell box only bounds the cells the exact membership test visits, so it is computed in
    // FP32 (FP64 runs at 1/64 rate here): its error (< 1e-6) is far inside the one-cell margin
    // (2/N), and the far-side cull keeps a 1e-4 rad margin.
    const float pi_f = 3.14159265358979f;
    const float af = asinf(fminf((float)r, 1.0f));
    const float bx = acosf(fmaxf(-1.0f, fminf(1.0f, o.Pf[0])));
    const float by = acosf(fmaxf(-1.0f, fminf(1.0f, o.Pf[1])));
    const float bz = acosf(fmaxf(-1.0f, fminf(1.0f, o.Pf[2])));
    const float xhi = cosf(fmaxf(0.0f, bx - af)), xlo = cosf(fminf(pi_f, bx + af));
    const float yhi = cosf(fmaxf(0.0f, by - af)), ylo = cosf(fminf(pi_f, by + af));
    const float Nf = (float)N;
    int i0 = (int)floorf((xlo * Nf + Nf - 1.0f) * 0.5f) - 1, i1 = (int)ceilf((xhi * Nf + Nf - 1.0f) * 0.5f) + 1;
    int j0 = (int)floorf((ylo * Nf + Nf - 1.0f) * 0.5f) - 1, j1 = (int)ceilf((yhi * Nf + Nf - 1.0f) * 0.5f) + 1;
    i0 = max(i0, 0); j0 = max(j0, 0); i1 = min(i1, N - 1); j1 = min(j1, N - 1);
    if (bz - af > 0.5f * pi_f + 1e-4f) i1 = i0 - 1;     // cap entirely on the far side
    o.box[0] = i0; o.box[1] = i1; o.box[2] = j0; o.box[3] = j1;
    return o;
}

// True when cell (i, j) lies in an earlier region's box (each cell is visited once, from the
// first box that holds it).
__device__ __forceinline__ bool in_earlier_box(const RegionGeo* sg, int r, int i, int j) {
    bool dup = false;
    for (int q = 0; q < r; q++)
        if (i >= sg[q].box[0] && i <= sg[q].box[1] && j >= sg[q].box[2] && j <= sg[q].box[3]) dup = true;
    return dup;
}

// InfoMap owner of a visible cell: a cell (x, y, mu) belongs to a region iff
// (x, y, mu) . P >= sqrt(1 - r^2); the last region in list order that contains it owns it
// (-1: none).  An FP32 test decides cells farther than 2e-6 from the edge (its error is below
// 1e-6); the others are decided by the explicitly rounded FP64 sequence, on the cell centres
// (2 i + 1 - N) / N of the table cellx (IEEE-divided once, as the oracle divides).
// float(v) for |v| < 2^22 without a conversion instruction: the bits 0x4B400000 + v are the float
// 2^23 + 2^22 + v exactly, and one subtraction leaves v.
__device__ __forceinline__ float small_int_to_float(int v) {
    return __int_as_float(0x4B400000 + v) - 12582912.0f;
}

// Box cells in the order t = 0, 1, ... (row-major, width w) for a thread that starts at t0 and
// steps by `step`: the quotient and remainder of the step are taken once, so the walk needs no
// division per cell.
struct BoxWalk {
    int row, col, dq, dr, w;
    __device__ __forceinline__ BoxWalk(int t0, int step, int width) : w(width) {
        row = t0 / width; col = t0 - row * width;
        dq = step / width; dr = step - dq * width;
    }
    __device__ __forceinline__ void next() {
        row += dq; col += dr;
        if (col >= w) { col -= w; row++; }
    }
};

__device__ __forceinline__ int cell_owner(const RegionGeo* sg, int n_regions, int N, float invN, int i, int j,
                                          float muf, const double* __restrict__ cell_mu, int64_t c,
                                          const double* __restrict__ cellx) {
    const float xf = small_int_to_float(2 * i + 1 - N) * invN, yf = small_int_to_float(2 * j + 1 - N) * invN;
    int owner = -1;
    for (int q = 0; q < n_regions; q++) {
        const float df = fmaf(xf, sg[q].Pf[0], fmaf(yf, sg[q].Pf[1], muf * sg[q].Pf[2]));
        bool in;
        if (df > sg[q].cosrf + 2e-6f) in = true;
        else if (df < sg[q].cosrf - 2e-6f) in = false;
        else {
            const double x = cellx[i];
            const double y = cellx[j];
            const double dot = __dadd_rn(__dadd_rn(__dmul_rn(x, sg[q].P[0]), __dmul_rn(y, sg[q].P[1])),
                                         __dmul_rn(cell_mu[c], sg[q].P[2]));
            in = dot >= sg[q].cosr;
        }
        if (in) owner = q;
    }
    return owner;
}

}  // namespace soap
