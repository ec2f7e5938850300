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

// Status word written by kernels (bounds checks that skip an access and record it).
enum DeviceFlag : unsigned int {
    kFlagTapRange = 1u,        // a cell's tap fell outside the precomputed kernel range
    kFlagBoxRange = 2u,        // a region box index left the grid
    kFlagJobOverflow = 4u      // a job table would overflow its capacity
};

}  // namespace soap

struct soap_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;

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

    // quiet velocity kernels, fixed point [n_mu][n_taps]
    long long* kq_fixed = nullptr;
    long long* sum_I_fixed = nullptr;   // [0] sum of I (fixed point), [1] visible cells

    // scratch (grow-only)
    soap::DevBuf stage_in;      // host -> device staging of spectra
    soap::DevBuf fq;            // quiet spectrum (fp64 or fp32) for Eq. 4
    soap::DevBuf contrast;      // [n_class][n_px] fp64 + fp32
    soap::DevBuf kphase;        // fixed-point kernels [n_phases][n_class][n_mu][n_taps]
    soap::DevBuf jobs;          // job tables
    soap::DevBuf coefs;         // job coefficients (fp64 and fp32)
    soap::DevBuf regions;       // region parameters
    soap::DevBuf region_geo;    // region centres and boxes per (phase, region)
    soap::DevBuf phases;
    soap::DevBuf out_stage;     // device output when the caller wants host output
    soap::DevBuf partial;       // direct-form and CCF partial sums
    soap::DevBuf ccf_tmp;       // CCF inputs / outputs
    soap::HostBuf host_stage;

    uint64_t launches = 0;

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
soap_status geometry_init(soap_ctx* c);                          // per-cell geometry + quiet kernels
soap_status pad_rows(soap_ctx* c, const double* src, double* dst64, float* dst32, int rows);

// Toeplitz quiet spectrum into dst (fp64 or fp32) on the context's stream.
soap_status toeplitz_quiet(soap_ctx* c, int precision, void* dst);
// Direct-form quiet spectrum.
soap_status direct_quiet(soap_ctx* c, int precision, void* dst);

struct RegionDev {      // one region as the kernels see it
    double lat_deg, lon_deg, radius, temp;
    int32_t type, cls;
};

// Active phases (Toeplitz) into dst [n_eff][n_phases][n_px].
soap_status toeplitz_active(soap_ctx* c, const RegionDev* regions_host, int n_regions,
                            const double* class_temp, const int* class_type, int n_class,
                            const double* phases_host, int n_phases, uint32_t effects,
                            int precision, void* dst);

soap_status rv_ccf_run(soap_ctx* c, const void* spectra_dev, int f32, int n_spec,
                       const double* mask_lambda, const double* mask_weight, int n_lines,
                       double width_kms, double v_lo, double v_step, int n_v, double* rv_dev,
                       double* fit_dev, double* ccf_dev);

}  // namespace soap
