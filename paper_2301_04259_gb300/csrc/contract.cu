// contract.cu -- Toeplitz form of the disk sum (quiet star, Alg. 1; active phases, Alg. 5
// with Eqs. 1-4) and the wavelength-dependent contrast (Sect. 4.3.1).
//
// Per phase p and region class (type, temperature) cl, the cells the class owns in the
// InfoMap add their two-tap kernels into per-mu-bin velocity kernels K[p][cl][b][k] (exact
// 64-bit fixed point).  With Q = sum_cl K (all active cells) the three effects of Eqs. 1-3,
// summed over cells and subtracted from the quiet integral (Eq. 4), are
//   TOT:   F_q - sum_b Q_b * S_q,b + sum_cl C_cl . sum_b K_cl,b * S_a(cl),b
//   FLUX:  F_q - sum_b Q_b * S_q,b + sum_cl C_cl . sum_b K_cl,b * S_q,b
//   BCONV: F_q - sum_b Q_b * S_q,b + sum_cl        sum_b K_cl,b * S_a(cl),b
// where "*" is the banded convolution (K * S)[m] = sum_k K[k] S[m-k] over the kernel's taps
// and C_cl(lambda) = B(lambda, T_cl) / B(lambda, T_quiet) multiplies on the common grid.
//
// A tap table lists, per (group, mu bin), the range of taps with non-zero kernel values in a
// block of PB consecutive phases; the contraction kernel reads the shifted row of each tap once
// and uses it for all PB phases.
#include <cmath>
#include <vector>

#include "contract_dev.cuh"

namespace soap {


// ---------------------------------------------------------------------------------------
// contrast (Sect. 4.3.1): C(lambda) = (exp(hc/lambda k T_q) - 1) / (exp(hc/lambda k T_a) - 1)
// ---------------------------------------------------------------------------------------
struct ClassTemps {
    double t[SOAP_MAX_CLASSES];
};

__global__ void k_contrast(int64_t n_px, double lam_s, double delta, double t_quiet, int n_class,
                           ClassTemps temps, double* c64, float* c32) {
    const double hck = kPlanckH * kLightSI / kBoltzmann * 1e10;   // Angstrom Kelvin
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n_px;
         m += (int64_t)gridDim.x * blockDim.x) {
        double lam = lam_s * exp((double)m * delta);
        double xq = expm1(hck / (lam * t_quiet));
        for (int cl = 0; cl < n_class; cl++) {
            double v = xq / expm1(hck / (lam * temps.t[cl]));
            c64[cl * n_px + m] = v;
            c32[cl * n_px + m] = (float)v;
        }
    }
}

// ---------------------------------------------------------------------------------------
// InfoMap + per-phase velocity kernels (Alg. 5)
// ---------------------------------------------------------------------------------------
// Region centre, cap and cell box per (phase, region), computed once (FP64 trigonometry).
// radii (optional, [n_phases][n_regions]): per-phase radii of evolving regions (Sect. 4.2.1).
__global__ void k_region_geo(int N, int n_regions, int n_phases, const RegionDev* regs,
                             const double* phases, double incl_deg, double alpha,
                             const double* __restrict__ radii, RegionGeo* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_phases * n_regions) return;
    const int p = t / n_regions, q = t % n_regions;
    RegionDev g = regs[q];
    if (radii) g.radius = radii[t];
    out[t] = region_geometry(N, g, phases[p], incl_deg, alpha);
}

// Blocks (phase p, split).  A visible cell (x, y, mu) belongs to a region iff
// (x, y, mu) . P >= sqrt(1 - r^2); the last region in list order that contains it owns it.  An
// FP32 test decides cells farther than 2e-6 from the edge (its error is below 1e-6); the others
// are decided by the explicitly rounded FP64 sequence.  Owned cells add their precomputed
// fixed-point contributions to the block's shared-memory kernels, which are then added to the
// phase's kernels with 64-bit atomics (exact, order-independent).
__global__ void k_phase_hist(int N, int n_regions, const RegionGeo* __restrict__ geo,
                             const double* __restrict__ cell_mu, const float* __restrict__ cell_mu32,
                             const int32_t* __restrict__ cell_j, const int32_t* __restrict__ cell_bin,
                             const long long* __restrict__ cell_k0, const long long* __restrict__ cell_k1,
                             int tap_min, int n_taps, int n_mu, int n_class, long long* kout,
                             int use_smem, int PB, double inv_scale, int fx_bits, int64_t row_len, int64_t pad,
                             long long* toff, int* gstart, double* c64, float* c32, int max_taps,
                             int* counters, int taps_smem, unsigned int* flags, int* bstart,
                             const double* __restrict__ cell_x, int mode) {
    __shared__ RegionGeo sg[SOAP_MAX_REGIONS];
    extern __shared__ long long hist_sm[];
    const int p = blockIdx.x;
    const int split = blockIdx.y, n_split = gridDim.y;
    const int nb = n_class * n_mu * n_taps;
    long long* gdst = kout + (int64_t)p * nb;
    long long* hist = use_smem ? hist_sm : gdst;
    if (threadIdx.x < n_regions) sg[threadIdx.x] = geo[(int64_t)p * n_regions + threadIdx.x];
    if (use_smem)
        for (int t = threadIdx.x; t < nb; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    const float invN = 1.0f / small_int_to_float(N);
    for (int r = 0; r < n_regions; r++) {
        const int i0 = sg[r].box[0], i1 = sg[r].box[1], j0 = sg[r].box[2], j1 = sg[r].box[3];
        if (i1 < i0 || j1 < j0) continue;
        const int wdt = i1 - i0 + 1;
        const int area = wdt * (j1 - j0 + 1);                  // <= N^2 < 2^31
        const int t0 = split * (int)blockDim.x + (int)threadIdx.x, step = n_split * (int)blockDim.x;
        BoxWalk wk(t0, step, wdt);
        for (int t = t0; t < area; t += step, wk.next()) {
            const int i = i0 + wk.col, jj = j0 + wk.row;
            if (in_earlier_box(sg, r, i, jj)) continue;
            const int c = jj * N + i;                          // N^2 < 2^31
            const int b = cell_bin[c];
            if (b < 0) continue;
            const int owner = cell_owner(sg, n_regions, N, invN, i, jj, cell_mu32[c], cell_mu, c, cell_x);
            if (owner < 0) continue;
            const int kk = cell_j[c] - tap_min;
            if (kk < 1 || kk >= n_taps) { atomicOr(flags, kFlagTapRange); continue; }
            long long* h = hist + (sg[owner].cls * n_mu + b) * n_taps;
            atomicAdd((unsigned long long*)&h[kk], (unsigned long long)cell_k0[c]);
            atomicAdd((unsigned long long*)&h[kk - 1], (unsigned long long)cell_k1[c]);
        }
    }
    if (use_smem) {
        __syncthreads();
        for (int t = threadIdx.x; t < nb; t += blockDim.x)
            if (hist[t]) atomicAdd((unsigned long long*)&gdst[t], (unsigned long long)hist[t]);
    }
    // The last block to finish among those feeding a phase block builds its tap table
    // (counter ticket after a memory fence: every other block's sums are visible by then).
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    const int pbk = p / PB;
    if (threadIdx.x == 0) {
        const int np_pb = min(PB, (int)gridDim.x - pbk * PB);
        const int t = atomicAdd(&counters[pbk], 1);
        s_last = t == np_pb * n_split - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        build_taps_dev(kout, pbk, (int)gridDim.x, n_class, n_mu, n_taps, tap_min, PB, mode, inv_scale, fx_bits, row_len,
                       pad, toff, gstart, c64, c32, max_taps, taps_smem ? hist_sm : nullptr, flags, bstart);
    }
}

// ---------------------------------------------------------------------------------------
// contraction
// ---------------------------------------------------------------------------------------
// One block: pixel tile blockIdx.x of phase block blockIdx.y, effect blockIdx.z.  Eight blocks
// per SM (at most 64 registers with 128 threads) keep the occupancy the tap loads need.
template <typename T, int PB, int R, int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS == 128 ? 8 : 1)
k_contract(int64_t n_px, Rows<T> rows, const long long* __restrict__ toff, const int* __restrict__ gstart,
           int G, int max_taps, const T* __restrict__ coefs, ClassTypes ctype, const T* __restrict__ contrast,
           const T* __restrict__ fq, int n_phases, EffectList effs, T* __restrict__ out,
           const int* __restrict__ bstart, int n_mu, int fold) {
    // a kernel launched after this one with an early start (the tensor-core CCF) may begin once
    // every CTA here has started: it waits for this grid before it reads the output
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int pb = blockIdx.y;
    const int np = min(PB, n_phases - pb * PB);
    T* out_rows = out + (int64_t)blockIdx.z * n_phases * n_px + (int64_t)pb * PB * n_px;
    const TableContrast<T> con{contrast, n_px, ctype};
    if (fold) {
        const long long* tt = toff + (int64_t)pb * max_taps;
        const int* gs = gstart + (int64_t)pb * (G + 1);
        const T* cb = coefs + (int64_t)pb * max_taps * PB;
        const int eff = effs.e[blockIdx.z];
        if constexpr (sizeof(T) == 4 && R % 2 == 0) {
            if (eff == SOAP_EFFECT_FLUX)
                contract_tile_fold32<PB, R, THREADS, SOAP_EFFECT_FLUX>(n_px, rows, tt, gs, G, cb, con, fq, blockIdx.x, np,
                                                                       out_rows);
            else if (eff == SOAP_EFFECT_BCONV)
                contract_tile_fold32<PB, R, THREADS, SOAP_EFFECT_BCONV>(n_px, rows, tt, gs, G, cb, con, fq, blockIdx.x, np,
                                                                        out_rows);
            else
                contract_tile_fold32<PB, R, THREADS, SOAP_EFFECT_TOT>(n_px, rows, tt, gs, G, cb, con, fq, blockIdx.x, np,
                                                                      out_rows);
        } else {
            contract_tile_fold<T, PB, R, THREADS>(n_px, rows, tt, gs, G, cb, con, fq, eff, blockIdx.x, np, out_rows);
        }
        return;
    }
    contract_tile<T, PB, R, THREADS>(n_px, rows, toff + (int64_t)pb * max_taps, gstart + (int64_t)pb * (G + 1), G,
                                     coefs + (int64_t)pb * max_taps * PB, con, fq, effs.e[blockIdx.z], blockIdx.x,
                                     np, out_rows, bstart ? bstart + (int64_t)pb * (G * n_mu + 1) : nullptr, n_mu);
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
static int grid_cap(int64_t n, int threads, int cap) {
    int64_t g = (n + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

template <typename T, int PB, int R, int THREADS>
static soap_status launch_contract(soap_ctx* c, int n_blocks, int G, int max_taps,
                                   const long long* toff, const int* gstart, const T* coefs,
                                   const ClassTypes& ct, const T* contrast, const T* fq,
                                   int n_phases, const EffectList& el, int n_eff, T* out,
                                   const T* q, const T* a0, const T* a1, const int* bstart = nullptr,
                                   int fold = 0) {
    Rows<T> rows;
    rows.q = q; rows.a[0] = a0; rows.a[1] = a1;
    int64_t tiles = (c->n_px + (int64_t)THREADS * R - 1) / ((int64_t)THREADS * R);
    dim3 grid((unsigned)tiles, (unsigned)n_blocks, (unsigned)n_eff);
    SOAP_TIMED(c, fq ? SOAP_TIMER_CONTRACT : SOAP_TIMER_CONTRACT_QUIET,
               k_contract<T, PB, R, THREADS><<<grid, THREADS, 0, c->stream>>>(
                   c->n_px, rows, toff, gstart, G, max_taps, coefs, ct, contrast, fq, n_phases, el, out,
                   bstart, c->n_mu, fold);
               SOAP_LAUNCHED(c));
    return SOAP_OK;
}

// Phase-block sizes and pixels per thread of the two precisions.
// (build-time overrides exist for measuring other tile shapes)
#ifndef SOAP_PB32
#define SOAP_PB32 4
#endif
#ifndef SOAP_R32
#define SOAP_R32 4
#endif
constexpr int kPB64 = 4, kR64 = 2, kT64 = 128;
constexpr int kPB32 = SOAP_PB32, kR32 = SOAP_R32, kT32 = 128;

// tap-table + coefficient scratch for a kernel set kfix with n_phases "phases" in blocks of PB
static soap_status tap_buffers(soap_ctx* c, int n_phases, int n_class, int PB, int mode, long long** toff,
                               int** gstart, double** c64, float** c32, int* n_blocks, int* G, int* max_taps,
                               int** bstart = nullptr) {
    *G = mode == 0 ? 1 : (mode == 1 ? 1 + n_class : n_class);
    *n_blocks = (n_phases + PB - 1) / PB;
    *max_taps = *G * c->n_mu * c->n_taps;
    size_t tb = (size_t)*n_blocks * *max_taps * sizeof(long long);
    size_t gb = (size_t)*n_blocks * (*G + 1) * sizeof(int);
    size_t off_g = (tb + 255) / 256 * 256;
    size_t off_b = (off_g + gb + 255) / 256 * 256;
    size_t bb = bstart ? (size_t)*n_blocks * (*G * c->n_mu + 1) * sizeof(int) : 0;
    SOAP_TRY(ensure(c->jobs, off_b + bb));
    if (bstart) *bstart = (int*)(c->jobs.as<char>() + off_b);
    size_t cb64 = (size_t)*n_blocks * *max_taps * PB * sizeof(double);
    size_t off32 = (cb64 + 255) / 256 * 256;
    SOAP_TRY(ensure(c->coefs, off32 + (size_t)*n_blocks * *max_taps * PB * sizeof(float)));
    *toff = c->jobs.as<long long>();
    *gstart = (int*)(c->jobs.as<char>() + off_g);
    *c64 = c->coefs.as<double>();
    *c32 = (float*)(c->coefs.as<char>() + off32);
    return SOAP_OK;
}

// Quiet integral (Alg. 1) in FP32 from the quiet taps as aligned groups (build_taps_dev): a thread
// owns 4 consecutive pixels; the taps of a group sit at row offsets 4q + e, e < 4, so their row
// values for the 4 pixels are 8 values from 4q + m0, two aligned 16-byte loads.  Groups are taken
// kQG at a time (all their loads issued before the first is applied: with ~50 groups and one
// thread per 4 pixels, ~10 warps per SM, the kernel is bound by the number of load round trips);
// per pixel the taps are added in table order, as in contract_tile (same results).
constexpr int kQG = 8;
__global__ void __launch_bounds__(128, 4)
k_quiet_groups(int64_t n_px, const float* __restrict__ q, const TapGroup* __restrict__ grp,
               const int* __restrict__ gstart, const float* __restrict__ coef, float* __restrict__ out) {
    const int64_t m0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (m0 >= n_px) return;
    const int n = gstart[1];
    const float* base = q + m0;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int i0 = 0; i0 < n; i0 += kQG) {
        TapGroup d[kQG];
        float W[kQG][8];
#pragma unroll
        for (int j = 0; j < kQG; j++) d[j] = grp[min(i0 + j, n - 1)];
#pragma unroll
        for (int j = 0; j < kQG; j++) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(base + d[j].off4));
            const float4 b = __ldg(reinterpret_cast<const float4*>(base + d[j].off4) + 1);
            W[j][0] = a.x; W[j][1] = a.y; W[j][2] = a.z; W[j][3] = a.w;
            W[j][4] = b.x; W[j][5] = b.y; W[j][6] = b.z; W[j][7] = b.w;
        }
        // selects instead of branches, so that no load is deferred to its use
#pragma unroll
        for (int j = 0; j < kQG; j++) {
            const int mk = i0 + j < n ? d[j].mask : 0;
#pragma unroll
            for (int e = 3; e >= 0; e--) {                     // offsets falling: table order
                const bool on = (mk >> e) & 1;
                const float cv = on ? __ldg(coef + d[j].tap0 - e) : 0.0f;
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const float t = fmaf(cv, W[j][e + r], acc[r]);
                    acc[r] = on ? t : acc[r];
                }
            }
        }
    }
    if ((n_px & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
        *reinterpret_cast<float4*>(out + m0) = make_float4(acc[0], acc[1], acc[2], acc[3]);
    } else {
#pragma unroll
        for (int r = 0; r < 4; r++)
            if (m0 + r < n_px) out[m0 + r] = acc[r];
    }
}

soap_status toeplitz_quiet(soap_ctx* c, int precision, void* dst) {
    // tap table built by the geometry kernel
    SOAP_TRY(join_geometry(c));
    const int nbk = 1, G = 1, mt = c->n_mu * SOAP_MAX_TAPS;
    ClassTypes ct{};
    EffectList el{{SOAP_EFFECT_TOT, 0, 0}};
    if (precision == SOAP_FP64)
        return launch_contract<double, 1, 1, 128>(c, nbk, G, mt, c->qtoff, c->qgstart, c->qc64, ct, nullptr,
                                                 nullptr, 1, el, 1, (double*)dst, c->q64, nullptr, nullptr);
    const unsigned blocks = (unsigned)((c->n_px + 4 * 128 - 1) / (4 * 128));
    SOAP_TIMED(c, SOAP_TIMER_CONTRACT_QUIET,
               k_quiet_groups<<<blocks, 128, 0, c->stream>>>(c->n_px, c->q32, c->qgrp, c->qgrp_start, c->qc32,
                                                            (float*)dst);
               SOAP_LAUNCHED(c));
    return SOAP_OK;
}

soap_status toeplitz_active(soap_ctx* c, const RegionDev* regions_host, int n_regions,
                            const double* class_temp, const int* class_type, int n_class,
                            const double* phases_host, int n_phases, uint32_t effects,
                            int precision, void* dst,
                            const double* radii_host) {
    const bool f64 = precision == SOAP_FP64;
    const size_t esz = f64 ? 8 : 4;
    const int ncl = n_class > 0 ? n_class : 1;
    // the main stream's position now: the previous call's contraction, the last reader of the
    // tap tables that this call's per-phase kernels rewrite, is before it
    SOAP_CUDA(cudaEventRecord(c->ev_main, c->stream));
    SOAP_TRY(ensure(c->fq, (size_t)c->n_px * esz));
    // contrast per class, or per (class, mu bin) with mu-dependent facula temperatures
    bool has_fac = false;
    for (int k = 0; k < n_class; k++) has_fac |= class_type[k] == SOAP_FACULA;
    const bool per_bin = c->facula_mu && has_fac;
    const int n_rows = per_bin ? ncl * c->n_mu : ncl;
    size_t cbytes = (size_t)n_rows * c->n_px;
    size_t off32 = (cbytes * 8 + 255) / 256 * 256;
    SOAP_TRY(ensure(c->contrast, off32 + cbytes * 4));
    double* con64 = c->contrast.as<double>();
    float* con32 = (float*)(c->contrast.as<char>() + off32);
    if (per_bin) {
        // facula rows: T_quiet + dT_f(mu_b), dT_f(mu) = 250.9 - 407.7 mu + 190.9 mu^2 (Sect. 4.3.1,
        // SOAP 2.0's limb brightening); spot rows repeat the class temperature
        const double hck = kPlanckH * kLightSI / kBoltzmann * 1e10;
        std::vector<double> temps((size_t)n_rows);
        std::vector<float> a32((size_t)n_rows);
        for (int k = 0; k < n_class; k++)
            for (int b = 0; b < c->n_mu; b++) {
                const double mu = c->mu_values[b];
                const double t = class_type[k] == SOAP_FACULA ? c->t_quiet + (250.9 - 407.7 * mu + 190.9 * mu * mu)
                                                              : class_temp[k];
                temps[(size_t)k * c->n_mu + b] = t;
                a32[(size_t)k * c->n_mu + b] = (float)(hck / (c->lam_s * t));
            }
        SOAP_TRY(ensure(c->contrast_t, (size_t)n_rows * (sizeof(double) + sizeof(float)) + 256));
        double* t_dev = c->contrast_t.as<double>();
        float* a_dev = reinterpret_cast<float*>(c->contrast_t.as<char>() + ((size_t)n_rows * 8 + 255) / 256 * 256);
        SOAP_TRY(upload_small(c, t_dev, temps.data(), temps.size() * sizeof(double)));
        SOAP_TRY(upload_small(c, a_dev, a32.data(), a32.size() * sizeof(float)));
        dim3 cgrid((unsigned)grid_cap(c->n_px, 256, 152 * 2), (unsigned)std::min(n_rows, 16));
        if (f64)
            SOAP_TIMED(c, SOAP_TIMER_CONTRAST,
                       k_contrast_rows<<<cgrid, 256, 0, c->stream>>>(c->n_px, c->lam_s, c->delta, c->t_quiet, n_rows,
                                                                     t_dev, con64, con32);
                       SOAP_LAUNCHED(c));
        else
            SOAP_TIMED(c, SOAP_TIMER_CONTRAST,
                       k_contrast_rows32<<<cgrid, 256, 0, c->stream>>>(
                           c->n_px, (float)(hck / (c->lam_s * c->t_quiet)), (float)c->delta, n_rows, a_dev, con32);
                       SOAP_LAUNCHED(c));
    } else if (n_class > 0) {
        ClassTemps tt{};
        ClassConsts cc{};
        const double hck = kPlanckH * kLightSI / kBoltzmann * 1e10;
        for (int k = 0; k < n_class; k++) {
            tt.t[k] = class_temp[k];
            cc.a[k] = (float)(hck / (c->lam_s * class_temp[k]));
        }
        if (f64)
            SOAP_TIMED(c, SOAP_TIMER_CONTRAST,
                       k_contrast<<<grid_cap(c->n_px, 256, 152 * 8), 256, 0, c->stream>>>(
                           c->n_px, c->lam_s, c->delta, c->t_quiet, n_class, tt, con64, con32);
                       SOAP_LAUNCHED(c));
        else
            SOAP_TIMED(c, SOAP_TIMER_CONTRAST,
                       k_contrast32<<<grid_cap(c->n_px, 256, 152 * 8), 256, 0, c->stream>>>(
                           c->n_px, (float)(hck / (c->lam_s * c->t_quiet)), (float)c->delta, n_class, cc, con32);
                       SOAP_LAUNCHED(c));
    }
    // regions and phases to the device (through the pinned ring: no wait for the stream), the
    // clears and the region boxes run on aux2, after the previous call's per-phase kernels (the
    // last readers of these buffers), overlapping the main stream's padded rows and contrast
    SOAP_CUDA(cudaStreamWaitEvent(c->aux2, c->ev_ph, 0));
    OnStream on2(c, c->aux2);
    size_t rbytes = (size_t)(n_regions > 0 ? n_regions : 1) * sizeof(RegionDev);
    size_t pbytes = (size_t)n_phases * sizeof(double);
    SOAP_TRY(ensure(c->regions, rbytes));
    SOAP_TRY(ensure(c->phases, pbytes));
    if (n_regions > 0)
        SOAP_TRY(upload_small(c, c->regions.p, regions_host, (size_t)n_regions * sizeof(RegionDev)));
    const double* radii_dev = nullptr;
    if (radii_host && n_regions > 0) {
        const size_t rb = (size_t)n_phases * n_regions * sizeof(double);
        SOAP_TRY(ensure(c->radii, rb));
        SOAP_TRY(upload_small(c, c->radii.p, radii_host, rb));
        radii_dev = c->radii.as<double>();
    }
    SOAP_TRY(upload_small(c, c->phases.p, phases_host, pbytes));
    // per-phase fixed-point kernels
    int64_t nb = (int64_t)ncl * c->n_mu * c->n_taps;
    size_t kbytes = (size_t)n_phases * nb * sizeof(long long);
    SOAP_TRY(ensure(c->kphase, kbytes));
    long long* kfix = c->kphase.as<long long>();
    // tap tables are built by the last block of each phase block (fused into k_phase_hist)
    const int PB = f64 ? kPB64 : kPB32;
    long long* toff; int* gstart; double* c64; float* c32; int nbk, G, mt; int* bstart = nullptr;
    // tables without the quiet group (mode 2: the contraction folds the quiet rows into the classes'
    // operands) unless the contrast has a row per mu bin (mode 1, per-bin folds)
    const int tmode = per_bin ? 1 : 2;
    SOAP_TRY(tap_buffers(c, n_phases, ncl, PB, tmode, &toff, &gstart, &c64, &c32, &nbk, &G, &mt,
                         per_bin ? &bstart : nullptr));
    SOAP_TRY(ensure(c->job_counters, (size_t)nbk * sizeof(int)));
    SOAP_CUDA(cudaMemsetAsync(c->job_counters.p, 0, (size_t)nbk * sizeof(int), c->stream));
    const size_t hist_bytes = (size_t)nb * sizeof(long long);
    const size_t kslice_bytes = (size_t)PB * nb * sizeof(long long);
    const int use_smem = hist_bytes <= 160 * 1024;
    const int taps_smem = kslice_bytes <= 96 * 1024;
    size_t smem = std::max(use_smem ? hist_bytes : (size_t)0, taps_smem ? kslice_bytes : (size_t)0);
    SOAP_CUDA(cudaMemsetAsync(kfix, 0, kbytes, c->stream));
    SOAP_TRY(fit_dynamic_smem(k_phase_hist, smem));
    // region centres and boxes per (phase, region)
    SOAP_TRY(ensure(c->region_geo, (size_t)n_phases * (n_regions > 0 ? n_regions : 1) * sizeof(RegionGeo)));
    if (n_regions > 0) {
        const int nt = n_phases * n_regions;
        SOAP_TIMED(c, SOAP_TIMER_REGIONS,
                   k_region_geo<<<(nt + 31) / 32, 32, 0, c->stream>>>(   // FP64 trig: spread over SMs
                       c->N, n_regions, n_phases, c->regions.as<RegionDev>(), c->phases.as<double>(), c->incl_deg,
                       c->alpha, radii_dev, c->region_geo.as<RegionGeo>());
                   SOAP_LAUNCHED(c));
    }
    SOAP_CUDA(cudaEventRecord(c->ev_rg, c->stream));
    c->stream = on2.saved;                                 // back to the main stream
    // split each phase over several blocks so that all SMs take part
    const int n_split = (int)std::max<int64_t>(1, std::min<int64_t>(8, (4 * 152 + n_phases - 1) / n_phases));
    dim3 hgrid((unsigned)n_phases, (unsigned)n_split);
    // the per-phase kernels run on the auxiliary stream (after the geometry queued there, the
    // region boxes and the previous contraction) while the main stream integrates the quiet star
    SOAP_CUDA(cudaStreamWaitEvent(c->aux, c->ev_rg, 0));
    SOAP_CUDA(cudaStreamWaitEvent(c->aux, c->ev_main, 0));
    {
        OnStream on(c, c->aux);
        SOAP_TIMED(c, SOAP_TIMER_PHASE_HIST,
                   k_phase_hist<<<hgrid, 256, smem, c->stream>>>(
                       c->N, n_regions, c->region_geo.as<RegionGeo>(), c->cell_mu, c->cell_mu32, c->cell_j,
                       c->cell_bin, c->cell_k0, c->cell_k1, c->tap_min, c->n_taps, c->n_mu, ncl, kfix,
                       use_smem, PB, std::ldexp(1.0, -c->fx_bits), c->fx_bits, c->row_len, c->pad, toff, gstart, c64,
                       c32, mt, c->job_counters.as<int>(), taps_smem, c->flags, bstart, c->cell_x, tmode);
                   SOAP_LAUNCHED(c));
        SOAP_CUDA(cudaEventRecord(c->ev_ph, c->stream));
    }
    // quiet integral for Eq. 4 in the output precision (joins the geometry), then the tap tables
    SOAP_TRY(toeplitz_quiet(c, precision, c->fq.p));
    SOAP_CUDA(cudaStreamWaitEvent(c->stream, c->ev_ph, 0));
    ClassTypes ct{};
    for (int k = 0; k < n_class; k++) ct.t[k] = class_type[k];
    EffectList el{{0, 0, 0}};
    int n_eff = 0;
    if (effects & SOAP_EFFECT_TOT) el.e[n_eff++] = SOAP_EFFECT_TOT;
    if (effects & SOAP_EFFECT_FLUX) el.e[n_eff++] = SOAP_EFFECT_FLUX;
    if (effects & SOAP_EFFECT_BCONV) el.e[n_eff++] = SOAP_EFFECT_BCONV;
    const double* a64s = c->active_set[0] ? c->a64[0] : c->a64[1];
    const double* a64f = c->active_set[1] ? c->a64[1] : c->a64[0];
    const float* a32s = c->active_set[0] ? c->a32[0] : c->a32[1];
    const float* a32f = c->active_set[1] ? c->a32[1] : c->a32[0];
    if (precision == SOAP_BF16X3) {
        // operand windows by TMA and one accumulator per class; a contrast row per mu bin (facula
        // limb brightening) or a shape beyond that form's limits takes the operand-building kernel
        if (!per_bin && toeplitz_tma_fits(c, ncl))
            return toeplitz_tma(c, kfix, n_phases, ncl, class_type, a32s, a32f, con32, el.e, n_eff, (float*)dst);
        return toeplitz_tc(c, kfix, n_phases, ncl, class_type, a32s, a32f, con32, per_bin, el.e, n_eff, (float*)dst);
    }
    if (f64)
        return launch_contract<double, kPB64, kR64, kT64>(c, nbk, G, mt, toff, gstart, c64, ct, con64,
                                                         c->fq.as<double>(), n_phases, el, n_eff,
                                                         (double*)dst, c->q64, a64s, a64f, bstart, tmode == 2);
    return launch_contract<float, kPB32, kR32, kT32>(c, nbk, G, mt, toff, gstart, c32, ct, con32,
                                                    c->fq.as<float>(), n_phases, el, n_eff,
                                                    (float*)dst, c->q32, a32s, a32f, bstart, tmode == 2);
}

}  // namespace soap
