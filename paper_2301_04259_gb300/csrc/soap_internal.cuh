// soap_internal.cuh -- context, error handling and shared device helpers of libsoap.
//
// The context owns all device memory.  Geometry lives on the full N x N grid (index
// j*N + i); local spectra are stored as replicate-padded rows so that every tap offset of a
// velocity kernel reads inside the row (the padding reproduces the "repeat the end value"
// edge rule of the interpolation exactly).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "soap.h"

namespace soap {

constexpr double kCKms = 299792.458;                 // km/s
constexpr double kPi = 3.14159265358979323846;
// Planck: h c / k_B from the exact SI values, in Angstrom Kelvin.
constexpr double kPlanckH = 6.62607015e-34;
constexpr double kLightSI = 299792458.0;
constexpr double kBoltzmann = 1.380649e-23;

// error reporting (thread-local last error)
void set_error(const char* fmt, ...);
void clear_error();

#define SOAP_TRY(expr)                                   \
    do {                                                 \
        soap_status st__ = (expr);                       \
        if (st__ != SOAP_OK) return st__;                \
    } while (0)

#define SOAP_CUDA(expr)                                                                  \
    do {                                                                                 \
        cudaError_t e__ = (expr);                                                        \
        if (e__ != cudaSuccess) {                                                        \
            ::soap::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e__),  \
                              __FILE__, __LINE__);                                       \
            return SOAP_ECUDA;                                                           \
        }                                                                                \
    } while (0)

// Bracket the launches in __VA_ARGS__ with CUDA events when the context is profiling.
#define SOAP_TIMED(ctx, timer, ...)                                                      \
    do {                                                                                 \
        cudaEvent_t a__ = nullptr;                                                       \
        if ((ctx)->profiling) a__ = ::soap::timer_begin(ctx);                             \
        __VA_ARGS__;                                                                     \
        if ((ctx)->profiling) ::soap::timer_end(ctx, timer, a__);                         \
    } while (0)

#define SOAP_LAUNCHED(ctx)                                                               \
    do {                                                                                 \
        (ctx)->launches++;                                                               \
        cudaError_t e__ = cudaGetLastError();                                            \
        if (e__ != cudaSuccess) {                                                        \
            ::soap::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e__), \
                              __FILE__, __LINE__);                                       \
            return SOAP_ECUDA;                                                           \
        }                                                                                \
    } while (0)

// Grow-only device scratch buffer owned by the context.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    template <class T> T* as() const { return static_cast<T*>(p); }
};
soap_status ensure(DevBuf& b, size_t bytes);
void release(DevBuf& b);

// Pinned host staging buffer (grow-only).
struct HostBuf {
    void* p = nullptr;
    size_t bytes = 0;
};
soap_status ensure_host(HostBuf& b, size_t bytes);
void release_host(HostBuf& b);

// Pinned staging ring for small host -> device uploads (regions, phases, masks).  A copy from
// pageable memory makes the driver wait for the stream before it copies, which would stall a
// caller that enqueues step after step; through the ring the host only copies into pinned
// memory and enqueues a small kernel that reads it through its device mapping (no copy engine:
// a small upload must not queue behind a large one).  Each upload records an event; a range of
// the ring is rewritten only once the reads that last used it are done.
struct PinnedRing {
    unsigned char* p = nullptr;        // host address
    unsigned char* dev = nullptr;      // the same memory, as the device sees it
    size_t cap = 0, head = 0;
    struct Use { size_t lo, hi; cudaEvent_t ev; };
    std::vector<Use> pending;          // oldest first
    std::vector<cudaEvent_t> free_ev;
};
constexpr size_t kRingBytes = size_t(4) << 20;

// Status word written by kernels (bounds checks that skip an access and record it).
enum DeviceFlag : unsigned int {
    kFlagTapRange = 1u,        // a cell's tap fell outside the precomputed kernel range
    kFlagBoxRange = 2u,        // a region box index left the grid
    kFlagJobOverflow = 4u,     // a tap table would overflow its capacity
    kFlagOrder = 8u,           // bisector injection: moved positions not increasing
    kFlagTimeout = 16u         // a tensor-core kernel's bounded barrier wait gave up
};

// The taps of one (group, mu bin) of a tap table at row offsets 4q .. 4q + 3 (build_taps_dev).
struct TapGroup {
    long long off4;    // 4q: row offset of the group's first value (a multiple of 4)
    int tap0;          // tap index of offset 4q (offset 4q + e is tap tap0 - e)
    int mask;          // bit e: offset 4q + e is one of the taps
};

// CCF state of one user of the CCF (the single-star calls, or the batched form): line and
// velocity tables (kept while the mask and the velocity grid stay the same), the cached mask
// matrix of the tensor-core form, and per-call scratch (partial sums, CCF, scaled CCF).
struct CcfState {
    DevBuf tab, tmp, m;
    std::vector<double> mask_key;        // mask_lambda, mask_weight, then width
    double vel_key[3] = {0, 0, -1};      // v_lo, v_step, n_v
    bool lines_ok = false;
    bool sorted = false;
    bool m_ok = false;                   // tensor-core mask matrix built for the current tables
    bool m_fresh = false;                // ... by the last kernel queued (the CCF must not start early)
};

// How one CCF call runs (ccf_prepare), for n_spec spectra.
struct CcfPlan {
    int n_spec = 0, n_lines = 0, n_v = 0, f32 = 0;
    double v_lo = 0, v_step = 0, h = 0;
    bool windowed = false;
    int n_wgroups = 0, n_chunks = 0;
    int tile_np = 0, tile_blocks = 0, tile_lines = 0;
    int64_t tc_chunk = 0;
    int tc_smin = 0, tc_smax = 0;
    // device tables (in CcfState::tab) and scratch (in CcfState::tmp)
    int* U = nullptr; double* f64 = nullptr; float* f32t = nullptr; float* w32 = nullptr;
    int* valid = nullptr; double* w64 = nullptr;
    int* S = nullptr; double* g64 = nullptr; float* g32 = nullptr;
    double* part = nullptr; double* ccf = nullptr; double* y = nullptr;
};

}  // namespace soap

struct soap_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    // auxiliary stream for work that can overlap the main stream: the cell geometry (forked from
    // the main stream when a star is set or updated, joined by its readers through
    // join_geometry) and the per-phase kernels (joined before the contraction); aux2 runs the
    // region and phase uploads and the region boxes of an active-phase call, after the previous
    // call's per-phase kernels.  ev_*: fork point, geometry done, region boxes done, per-phase
    // kernels done, main stream at the start of an active-phase call.
    cudaStream_t aux = nullptr, aux2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_geo = nullptr, ev_rg = nullptr, ev_ph = nullptr, ev_main = nullptr;
    bool geo_pending = false;           // geometry queued on aux, not yet joined by the main stream

    // star
    int N = 0;
    int n_mu = 0;
    int64_t n_px = 0;
    double vsini = 0, incl_deg = 0, u1 = 0, u2 = 0, alpha = 0;
    double lam_s = 0, lam_e = 0, t_quiet = 0, delta = 0;
    double mu_values[SOAP_MAX_MU] = {};
    int mu_sorted = 0;      // mu_values strictly increasing (fast nearest-mu search)

    // velocity kernels: taps k = tap_min .. tap_min + n_taps - 1; padded rows
    int tap_min = 0;
    int n_taps = 0;
    int64_t pad = 0;        // replicate padding on each side of a row
    int64_t row_len = 0;    // padded row length (elements)
    int fx_bits = 0;        // fixed-point kernels: value = integer * 2^-fx_bits
    int64_t n_visible = 0;
    double total_I = 0;

    // per-cell geometry on the full grid (index j*N + i)
    double* cell_I = nullptr;      // limb-darkened weight (0 off disk)
    double* cell_w = nullptr;      // interpolation weight w
    double* cell_mu = nullptr;     // mu (0 off disk)
    int32_t* cell_j = nullptr;     // tap j = ceil(s)
    int32_t* cell_bin = nullptr;   // nearest-mu bin, -1 off disk
    float* cell_mu32 = nullptr;    // mu in FP32 (membership pre-test)
    long long* cell_k0 = nullptr;  // fixed-point I (1 - w), tap j
    long long* cell_k1 = nullptr;  // fixed-point I w, tap j - 1
    unsigned int* flags = nullptr; // device status word

    // local spectra, padded rows [n_mu][row_len]; element n at [pad + n]
    double* q64 = nullptr;
    float* q32 = nullptr;
    double* a64[2] = {nullptr, nullptr};   // [0] spot, [1] facula
    float* a32[2] = {nullptr, nullptr};
    bool active_set[2] = {false, false};
    bool facula_mu = false;                // facula temperature T_quiet + dT_f(mu) per mu bin
    bool ccf_tc = false;                   // soap_active_rv at SOAP_FP32: the CCF on the tensor cores
    bool q64_ok = false;                   // float64 rows hold the last quiet upload
    bool a64_ok[2] = {false, false};       // (a float32 upload fills the float32 rows only)

    // quiet velocity kernels, fixed point [n_mu][n_taps]
    long long* kq_fixed = nullptr;
    long long* sum_I_fixed = nullptr;   // [0] sum of I (fixed point), [1] visible cells
    // quiet tap table, rebuilt with the geometry: row offsets, group starts, coefficients
    long long* qtoff = nullptr;     // [n_mu * SOAP_MAX_TAPS]
    int* qgstart = nullptr;         // [2]
    soap::TapGroup* qgrp = nullptr; // quiet taps as aligned groups [n_mu * (SOAP_MAX_TAPS + 1)]
    int* qgrp_start = nullptr;      // [2]
    double* qc64 = nullptr;
    float* qc32 = nullptr;
    int* geo_counter = nullptr;
    double* cell_x = nullptr;          // [N] (2 i + 1 - N) / N, the cell centres' x (and y)

    // scratch (grow-only)
    soap::DevBuf stage_in;      // host -> device staging of spectra
    soap::DevBuf fq;            // quiet spectrum (fp64 or fp32) for Eq. 4
    soap::DevBuf contrast;      // [n_class][n_px] fp64 + fp32 (per (class, mu bin) rows with facula_mu)
    soap::DevBuf contrast_t;    // per-row temperatures / FP32 constants of the per-bin contrast
    soap::DevBuf kphase;        // fixed-point kernels [n_phases][n_class][n_mu][n_taps]
    soap::DevBuf jobs;          // tap tables (row offsets + group starts)
    soap::DevBuf coefs;         // tap coefficients (fp64 and fp32)
    soap::DevBuf job_counters;  // per phase block: blocks done (fused tap tables)
    soap::DevBuf regions;       // region parameters
    soap::DevBuf region_geo;    // region centres and boxes per (phase, region)
    soap::DevBuf phases;
    soap::DevBuf radii;         // per-(phase, region) radii of evolving regions
    soap::DevBuf out_stage;     // device output when the caller wants host output
    soap::DevBuf partial;       // direct-form partial sums
    // direct form: visible cells compacted once per geometry (direct.cu); geo_version counts
    // geometry computations
    soap::DevBuf dir_cells, dir_count, dir_rows;
    uint64_t geo_version = 0, dir_version = ~0ull, dir_rows_version = ~0ull;
    int dir_prec = -1;
    const void* dir_rows_src = nullptr;          // the rows dir_rows was shifted from
    soap::HostBuf host_stage;
    soap::PinnedRing ring;      // small uploads (see PinnedRing)

    // instrumental resolution (soap_set_instrument_resolution): taps [2K+1] in f64, then f32 at
    // lsf_off32; lsf_K < 0 when off; lsf_tmp holds spectra before the line-spread function
    double lsf_R = 0.0;
    int lsf_K = -1;
    size_t lsf_off32 = 0, lsf_offp64 = 0, lsf_offp32 = 0;
    soap::DevBuf lsf_taps, lsf_tmp;
    soap::DevBuf bis_tab;       // bisector tables of the last injection
    soap::DevBuf tc_coef;       // tensor-core contraction: kernel rows (BF16 hi / lo) + block flags
    // tensor-core contraction with TMA-loaded windows (toeplitz_tma.cu): the FP32 rows as BF16 hi / lo
    // planes of 8 mu bins per pixel, rebuilt when the rows change (rows_version counts uploads)
    soap::DevBuf tm_planes, tm_coef;
    uint64_t rows_version = 0, tm_planes_version = ~0ull;
    const float* tm_planes_src[3] = {nullptr, nullptr, nullptr};

    // CCF of the single-star calls (soap_rv_ccf, soap_active_rv)
    soap::CcfState ccf;

    // host-transfer pipeline: uploads from host memory run on in_stream, downloads of host
    // results on out_stream, ordered against the compute stream by events.  up_* serve the
    // quiet / spot / facula uploads (filled: copy done; free: pad_rows has read the stage);
    // dn_* are two alternating device buffers for host results (spec / rv: the spectra /
    // the RVs are written; free: their copy to the host is done).
    bool host_async = false;            // calls with host outputs return before the copies end
    cudaStream_t in_stream = nullptr, out_stream = nullptr;
    soap::DevBuf up_stage[3];
    cudaEvent_t up_filled[3] = {}, up_free[3] = {};
    soap::DevBuf dn_stage[2];
    cudaEvent_t dn_spec[2] = {}, dn_rv[2] = {}, dn_free[2] = {};
    int dn_next = 0;

    uint64_t launches = 0;

    // batched form: grow-only buffers, the captured graph and the key of what it baked in
    soap::DevBuf b_items, b_regions, b_phases, b_phase_item, b_phase_block, b_pblocks, b_order;
    soap::DevBuf b_cellIfx, b_IB, b_colj, b_colw, b_kq, b_qtoff, b_qgs, b_qc32, b_fq;
    soap::DevBuf b_geo, b_kfix, b_counters, b_toff, b_gstart, b_coefs, b_ticket;
    cudaGraphExec_t b_graph_exec = nullptr;
    std::vector<uint64_t> b_graph_key;
    uint64_t b_graph_kernels = 0;
    int b_variant = -1;             // chosen by soap_batch_set_variant / the autotuner; -1: default
    // batched RVs (soap_batch_set_rv): mask and velocity grid, fit margin, CCF form, own CCF state
    bool b_rv_set = false;
    std::vector<double> b_rv_lambda, b_rv_weight;
    double b_rv_width = 0, b_rv_v_lo = 0, b_rv_v_step = 0, b_rv_margin = 0;
    int b_rv_n_v = 0, b_rv_tc = 0;
    soap::CcfState b_ccf;
    soap::DevBuf b_win;             // per phase: first point and length of its fit window

    // per-kernel timers
    bool profiling = false;
    struct TimedLaunch { int timer; cudaEvent_t a, b; };
    std::vector<TimedLaunch> pending;   // recorded, not yet folded into the totals
    std::vector<cudaEvent_t> event_pool; // free events
    double timer_ms[SOAP_TIMER_COUNT] = {};
    uint64_t timer_n[SOAP_TIMER_COUNT] = {};
};

namespace soap {

// timers (api.cu)
cudaEvent_t timer_begin(soap_ctx* c);
void timer_end(soap_ctx* c, int timer, cudaEvent_t begin);

// ---------------------------------------------------------------------------------------
// kernels and launchers implemented in the .cu files
// ---------------------------------------------------------------------------------------
// A launch may use 48 KB of shared memory, static and dynamic together, unless the kernel has
// opted in to more: opt in when the kernel's static part plus `dynamic` exceeds that.
template <typename Kernel>
inline soap_status fit_dynamic_smem(Kernel kernel, size_t dynamic) {
    cudaFuncAttributes a{};
    SOAP_CUDA(cudaFuncGetAttributes(&a, kernel));
    if (a.sharedSizeBytes + dynamic > 48 * 1024)
        SOAP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dynamic));
    return SOAP_OK;
}

soap_status geometry_init(soap_ctx* c);                          // per-cell geometry + quiet kernels (on aux)
soap_status join_geometry(soap_ctx* c);                          // main stream waits for a pending geometry

// Launches and timers inside the scope go to stream s instead of the context's main stream.
struct OnStream {
    soap_ctx* c;
    cudaStream_t saved;
    OnStream(soap_ctx* c_, cudaStream_t s) : c(c_), saved(c_->stream) { c->stream = s; }
    ~OnStream() { c->stream = saved; }
    OnStream(const OnStream&) = delete;
    OnStream& operator=(const OnStream&) = delete;
};
soap_status pad_rows(soap_ctx* c, const double* src, double* dst64, float* dst32, int rows);
soap_status pad_rows32(soap_ctx* c, const float* src, float* dst32, int rows);
// instrumental resolution (instrument.cu)
soap_status set_instrument(soap_ctx* c, double resolving_power);
soap_status launch_lsf(soap_ctx* c, const void* in, void* out, int f32, int64_t n_spec);
// bisector injection (convection.cu)
soap_status inject_bisectors(soap_ctx* c, const double* in, double* out, int n_rows, const double* bis_host,
                             const double* orig_host, int n_d);
// Copy `bytes` of host memory to device memory `dst` on the context stream through the pinned
// ring (pageable sources are fine; the source may change once the call returns).
soap_status upload_small(soap_ctx* c, void* dst, const void* src, size_t bytes);
void ring_release(soap_ctx* c);
// True when the CCF line tables of `st` were built from exactly this mask and width.
bool ccf_mask_same(const CcfState& st, const double* mask_lambda, const double* mask_weight,
                   int n_lines, double width_kms);

// Toeplitz quiet spectrum into dst (fp64 or fp32) on the context's stream.
soap_status toeplitz_quiet(soap_ctx* c, int precision, void* dst);
// Direct-form quiet spectrum.
soap_status direct_quiet(soap_ctx* c, int precision, void* dst);

struct RegionDev {      // one region as the kernels see it
    double lat_deg, lon_deg, radius, temp;
    int32_t type, cls;
};

// Active phases (Toeplitz) into dst [n_eff][n_phases][n_px].
// Active-phase contraction on the tensor cores (SOAP_BF16X3): kfix [n_phases][ncl][n_mu][n_taps]
// fixed-point kernels, FP32 rows / contrast / F_q of the context; out [n_eff][n_phases][n_px].
soap_status toeplitz_tc(soap_ctx* c, const long long* kfix, int n_phases, int ncl, const int* class_type,
                        const float* a_spot, const float* a_fac, const float* con32, bool per_bin,
                        const int* effects, int n_eff, float* out);
// The same contraction with the Toeplitz operand taken from TMA-loaded windows of BF16 planes and
// one accumulator per class (contrast applied at readout); SOAP_ERANGE when a limit of that form is
// exceeded (the caller then uses toeplitz_tc).
soap_status toeplitz_tma(soap_ctx* c, const long long* kfix, int n_phases, int ncl, const int* class_type,
                         const float* a_spot, const float* a_fac, const float* con32, const int* effects, int n_eff,
                         float* out);
bool toeplitz_tma_fits(const soap_ctx* c, int ncl);
soap_status toeplitz_active(soap_ctx* c, const RegionDev* regions_host, int n_regions,
                            const double* class_temp, const int* class_type, int n_class,
                            const double* phases_host, int n_phases, uint32_t effects,
                            int precision, void* dst,
                            const double* radii_host = nullptr);

// Batched form (batch.cu); variant in 0 .. batch_num_variants() - 1, out [n_phases][n_px] FP32
// (F, or F - F_q when residual).
// rv (nullable): device [n_phases] RVs of the output rows (needs the RV mask of soap_batch_set_rv).
soap_status batch_run(soap_ctx* c, const soap_batch_item* items, int n_items, const soap_region* regions,
                      int n_regions, const double* phases, int n_phases, int variant, int residual, float* out,
                      double* rv = nullptr);
int batch_num_variants();
int batch_default_variant(int max_phases_per_item);
void batch_variant_info(int v, int* phases_per_block, int* px_per_thread);
void batch_release(soap_ctx* c);

// CCF + Gaussian RV fit (Sect. 4.1) in two steps.  ccf_prepare makes the host decisions for
// n_spec spectra, sizes the scratch of `st` and, when the mask or the velocity grid changed,
// uploads the mask and builds the line / velocity tables (and, for the tensor-core form, the mask
// matrix) on the context's stream.  ccf_enqueue then only launches kernels (no allocation, no
// host transfer: it may be captured into a graph): partial sums, their reduction and the fits.
// tc: FP32 spectra whose CCF may run on the tensor cores (BF16 split, ccf_tc.cu) where that
// form applies (mask sorted by wavelength, at most 256 velocities).  win (nullable): per spectrum
// the first velocity index and the number of points of its fit window ([n_spec][2]).
soap_status ccf_prepare(soap_ctx* c, CcfState& st, const double* mask_lambda, const double* mask_weight,
                        int n_lines, double width_kms, double v_lo, double v_step, int n_v, int n_spec,
                        int f32, int tc, CcfPlan& p);
soap_status ccf_enqueue(soap_ctx* c, CcfState& st, const CcfPlan& p, const void* spectra_dev, double* rv_dev,
                        double* fit_dev, double* ccf_dev, const int* win);
// Both steps, for the single-star calls (the context's own CCF state).
soap_status rv_ccf_run(soap_ctx* c, const void* spectra_dev, int f32, int n_spec,
                       const double* mask_lambda, const double* mask_weight, int n_lines,
                       double width_kms, double v_lo, double v_step, int n_v, double* rv_dev,
                       double* fit_dev, double* ccf_dev, int tc = 0);
bool ccf_tc_fits(int n_v);
int64_t ccf_tc_chunk(int64_t n_px, int n_spec, int sms);
// Mask matrix of the tensor-core form for the tables of `st` (once per mask and grid).
soap_status ccf_tc_build_m(soap_ctx* c, CcfState& st, const CcfPlan& p);
soap_status ccf_tc(soap_ctx* c, CcfState& st, const CcfPlan& p, const float* spectra, float* partial);

}  // namespace soap

// K * 2^-bits rounded to the nearest float (ties to even) with integer operations only: the
// fixed-point kernels reach 2^61, and GB300 converts 64-bit integers through its (slow) FP64
// unit.  Valid for |K| < 2^63 and results in the normal float range.
__device__ __forceinline__ float fixed_to_float(long long K, int bits) {
    if (K == 0) return 0.0f;
    const unsigned int sign = K < 0 ? 0x80000000u : 0u;
    unsigned long long a = K < 0 ? (unsigned long long)(-K) : (unsigned long long)K;
    const int e = 63 - __clzll(a);                    // a in [2^e, 2^(e+1))
    unsigned int m;                                   // 24-bit significand with the hidden bit
    int ex = e;
    if (e <= 23) {
        m = (unsigned int)(a << (23 - e));
    } else {
        const int sh = e - 23;
        const unsigned long long q = a >> sh;
        const unsigned long long rem = a & ((1ull << sh) - 1ull);
        const unsigned long long half = 1ull << (sh - 1);
        m = (unsigned int)q;
        if (rem > half || (rem == half && (m & 1u))) {
            m++;
            if (m == (1u << 24)) { m >>= 1; ex++; }
        }
    }
    const int biased = ex - bits + 127;               // value = m 2^(ex - 23) 2^-bits
    return __uint_as_float(sign | ((unsigned int)biased << 23) | (m & 0x7FFFFFu));
}

// ---------------------------------------------------------------------------------------
// tap tables of the Toeplitz contraction (shared by geometry.cu, contract.cu and batch.cu)
// ---------------------------------------------------------------------------------------
namespace soap {

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


// K * 2^-bits rounded to the nearest float (ties to even) with integer operations only: the
// fixed-point kernels reach 2^61, and GB300 converts 64-bit integers through its (slow) FP64
// unit.  Valid for |K| < 2^63 and results in the normal float range.
__device__ __forceinline__ float fixed_to_float(long long K, int bits) {
    if (K == 0) return 0.0f;
    const unsigned int sign = K < 0 ? 0x80000000u : 0u;
    unsigned long long a = K < 0 ? (unsigned long long)(-K) : (unsigned long long)K;
    const int e = 63 - __clzll(a);                    // a in [2^e, 2^(e+1))
    unsigned int m;                                   // 24-bit significand with the hidden bit
    int ex = e;
    if (e <= 23) {
        m = (unsigned int)(a << (23 - e));
    } else {
        const int sh = e - 23;
        const unsigned long long q = a >> sh;
        const unsigned long long rem = a & ((1ull << sh) - 1ull);
        const unsigned long long half = 1ull << (sh - 1);
        m = (unsigned int)q;
        if (rem > half || (rem == half && (m & 1u))) {
            m++;
            if (m == (1u << 24)) { m >>= 1; ex++; }
        }
    }
    const int biased = ex - bits + 127;               // value = m 2^(ex - 23) 2^-bits
    return __uint_as_float(sign | ((unsigned int)biased << 23) | (m & 0x7FFFFFu));
}

// ---------------------------------------------------------------------------------------
// tap tables of the Toeplitz contraction
// ---------------------------------------------------------------------------------------
// A tap table lists, for one block of PB consecutive phases and each (group, mu bin), the taps k
// from the lowest to the highest with a non-zero kernel value in any of those phases, ordered by
// group, then bin, then k:
//   gstart[G+1]   first tap of each group (group 0: quiet rows; group g >= 1: class g-1)
//   toff[tap]     element offset bin * row_len + pad - k: the row value S_b[m - k] of pixel m
//                 is rows[toff + m]
//   coef[tap][PB] kernel value of each phase of the block (0 where a phase has none)
// kfix: [n_phases][n_class][n_mu][n_taps] in units of 2^-fx_bits (inv_scale = 2^-fx_bits).
// mode 0 (quiet): one group, +K of class 0.  mode 1 (active): group 0 = -sum_cl K (quiet rows),
// group g = +K of class g-1.  mode 2 (active, quiet rows folded into the classes' operands):
// group g = +K of class g.  Block pb covers phases pb*PB .. pb*PB+PB-1; its outputs start at
// toff + pb*max_taps,
// gstart + pb*(G+1) and coef + pb*max_taps*PB.  A table that would exceed max_taps is left
// empty and flags kFlagJobOverflow.
// agrp / agstart (optional): the same taps as aligned groups.  The taps of one (group, bin) are
// consecutive shifts of one row, at offsets o_hi, o_hi - 1, .., o_lo; aligned group q holds those
// of them in 4q .. 4q + 3 (TapGroup: off4 = 4q, the tap index of offset 4q, a bit per present
// offset; groups listed from the highest q down, like the taps), so that a contraction can read the row values of four consecutive pixels for all of
// a group's taps as two aligned 16-byte vectors.  agstart[g] is the first aligned group of
// group g (G + 1 entries, last = total); block pb's groups start at agrp + pb * max_groups with
// max_groups = max_taps + G n_mu (a (group, bin) with nk taps has at most nk + 1 groups).
__device__ __forceinline__ void build_taps_dev(const long long* __restrict__ kfix, int pb, int n_phases,
                                               int n_class, int n_mu, int n_taps, int tap_min, int PB, int mode,
                                               double inv_scale, int fx_bits, int64_t row_len, int64_t pad,
                                               long long* toff,
                                               int* gstart, double* c64, float* c32, int max_taps,
                                               long long* s_k, unsigned int* flags, int* bstart = nullptr,
                                               TapGroup* agrp = nullptr, int* agstart = nullptr) {
    __shared__ int s_lo[(1 + SOAP_MAX_CLASSES) * SOAP_MAX_MU];
    __shared__ int s_hi[(1 + SOAP_MAX_CLASSES) * SOAP_MAX_MU];
    __shared__ int s_off[(1 + SOAP_MAX_CLASSES) * SOAP_MAX_MU];
    __shared__ int s_goff[(1 + SOAP_MAX_CLASSES) * SOAP_MAX_MU];
    __shared__ int s_warp[32];
    __shared__ int s_total;
    const int use_smem = s_k != nullptr;
    const int G = mode == 0 ? 1 : (mode == 1 ? 1 + n_class : n_class);
    const int ngb = G * n_mu;
    const int p0 = pb * PB;
    const int np = min(PB, n_phases - p0);
    const int64_t nb = (int64_t)n_class * n_mu * n_taps;
    // the block's slice of kernels, [np][n_class][n_mu][n_taps], staged with coalesced loads
    const long long* src = kfix + (int64_t)p0 * nb;
    const long long* K = src;
    if (use_smem) {
        const int64_t n_el = (int64_t)np * nb;
        for (int64_t t0 = threadIdx.x; t0 < n_el; t0 += 8 * (int64_t)blockDim.x) {
            long long v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int64_t t = t0 + (int64_t)u * blockDim.x;
                v[u] = t < n_el ? __ldcg(src + t) : 0;      // written by other blocks' atomics
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int64_t t = t0 + (int64_t)u * blockDim.x;
                if (t < n_el) s_k[t] = v[u];
            }
        }
        __syncthreads();
        K = s_k;
    }
    auto kval = [&](const long long* q) -> long long { return use_smem ? *q : __ldcg(q); };
    auto value = [&](int g, int b, int pl, int kk) -> long long {
        if (pl >= np) return 0;
        const long long* base = K + (int64_t)pl * nb;
        if (g == 0 && mode == 1) {
            long long s = 0;
            for (int cl = 0; cl < n_class; cl++) s += kval(base + ((int64_t)cl * n_mu + b) * n_taps + kk);
            return -s;
        }
        const int cl = mode == 0 ? 0 : (mode == 1 ? g - 1 : g);
        return kval(base + ((int64_t)cl * n_mu + b) * n_taps + kk);
    };
    // tap range of each (group, bin) over the block's phases
    for (int t = threadIdx.x; t < ngb; t += blockDim.x) {
        const int g = t / n_mu, b = t % n_mu;
        int lo = n_taps, hi = -1;
        const int c0 = mode == 0 ? 0 : (mode == 2 ? g : (g == 0 ? 0 : g - 1));
        const int c1 = (mode == 1 && g == 0) ? n_class : c0 + 1;
        for (int pl = 0; pl < np; pl++) {
            const long long* base = K + (int64_t)pl * nb;
            for (int cl = c0; cl < c1; cl++) {
                const long long* row = base + ((int64_t)cl * n_mu + b) * n_taps;
                for (int kk = 0; kk < n_taps; kk++)
                    if (kval(row + kk) != 0) { lo = min(lo, kk); hi = max(hi, kk); }
            }
        }
        s_lo[t] = lo; s_hi[t] = hi;
    }
    // exclusive prefix sums (warp scans, chunks of blockDim.x) of the tap counts and of the
    // aligned-group counts per (group, bin)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t o_top = pad - tap_min;                       // offset of tap 0 in bin 0
    auto scan = [&](auto count, int* dst) -> int {
        if (threadIdx.x == 0) s_total = 0;
        __syncthreads();
        for (int c0 = 0; c0 < ngb; c0 += blockDim.x) {
            const int t = c0 + threadIdx.x;
            const int n = t < ngb ? count(t) : 0;
            int x = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_warp[warp] = x;
            __syncthreads();
            if (warp == 0) {
                int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, w, o);
                    if (lane >= o) w += y;
                }
                if (lane < nw) s_warp[lane] = w;
            }
            __syncthreads();
            if (t < ngb) dst[t] = s_total + (warp > 0 ? s_warp[warp - 1] : 0) + x - n;
            __syncthreads();
            if (threadIdx.x == 0) s_total += s_warp[nw - 1];
            __syncthreads();
        }
        return s_total;
    };
    auto n_groups = [&](int t) -> int {
        if (s_hi[t] < s_lo[t]) return 0;
        const int64_t ob = (int64_t)(t % n_mu) * row_len + o_top;
        return (int)(((ob - s_lo[t]) >> 2) - ((ob - s_hi[t]) >> 2) + 1);
    };
    const int total_groups = agrp ? scan(n_groups, s_goff) : 0;
    __syncthreads();
    const int total = scan([&](int t) { return s_hi[t] >= s_lo[t] ? s_hi[t] - s_lo[t] + 1 : 0; }, s_off);
    int* gs = gstart + (int64_t)pb * (G + 1);
    if (total > max_taps) {
        if (threadIdx.x == 0) atomicOr(flags, kFlagJobOverflow);
        for (int g = threadIdx.x; g <= G; g += blockDim.x) gs[g] = 0;
        if (agrp)
            for (int g = threadIdx.x; g <= G; g += blockDim.x) agstart[(int64_t)pb * (G + 1) + g] = 0;
        return;
    }
    for (int g = threadIdx.x; g <= G; g += blockDim.x) gs[g] = g < G ? s_off[g * n_mu] : total;
    if (agrp) {
        int* ags = agstart + (int64_t)pb * (G + 1);
        for (int g = threadIdx.x; g <= G; g += blockDim.x) ags[g] = g < G ? s_goff[g * n_mu] : total_groups;
    }
    // per-(group, bin) tap starts, for contractions that fold each bin separately
    if (bstart) {
        int* bs = bstart + (int64_t)pb * (ngb + 1);
        for (int t = threadIdx.x; t <= ngb; t += blockDim.x) bs[t] = t < ngb ? s_off[t] : total;
    }
    // row offsets and coefficients [tap][PB]: one warp per (group, bin)
    for (int t = warp; t < ngb; t += nw) {
        if (s_hi[t] < s_lo[t]) continue;
        const int g = t / n_mu, b = t % n_mu;
        const int nk = s_hi[t] - s_lo[t] + 1;
        const int64_t tap0 = (int64_t)pb * max_taps + s_off[t];
        for (int kk = lane; kk < nk; kk += 32)
            toff[tap0 + kk] = (int64_t)b * row_len + pad - (tap_min + s_lo[t] + kk);
        if (agrp) {
            // taps kk = 0 .. nk-1 at offsets o_hi - kk (tap index within the block: s_off[t] + kk)
            const int64_t o_hi = (int64_t)b * row_len + o_top - s_lo[t], o_lo = o_hi - (nk - 1);
            const int64_t q_hi = o_hi >> 2;
            const int ng = (int)(q_hi - (o_lo >> 2) + 1);
            TapGroup* dst = agrp + (int64_t)pb * (max_taps + ngb) + s_goff[t];
            for (int i = lane; i < ng; i += 32) {               // table order: offsets falling
                const int64_t off4 = 4 * (q_hi - i);
                int mask = 0;
                for (int e = 0; e < 4; e++)
                    if (off4 + e >= o_lo && off4 + e <= o_hi) mask |= 1 << e;
                TapGroup tg;
                tg.off4 = off4;
                tg.tap0 = s_off[t] + (int)(o_hi - off4);
                tg.mask = mask;
                dst[i] = tg;
            }
        }
        for (int e = lane; e < nk * PB; e += 32) {
            const int kk = e / PB, pl = e % PB;
            const long long K = value(g, b, pl, s_lo[t] + kk);
            if (c64) c64[tap0 * PB + e] = (double)K * inv_scale;
            c32[tap0 * PB + e] = fixed_to_float(K, fx_bits);
        }
    }
}

}  // namespace soap
