// api.cu -- C-ABI entry points of libsoap: argument validation, context and memory
// management, host<->device staging.  All arithmetic of the method runs in the kernels of
// geometry.cu, contract.cu, direct.cu and ccf.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "soap_internal.cuh"

namespace soap {

static thread_local char g_error[1024];

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_error, sizeof(g_error), fmt, ap);
    va_end(ap);
}

void clear_error() { g_error[0] = '\0'; }

soap_status ensure(DevBuf& b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return SOAP_OK;
    if (b.p) {
        // the old buffer may still be read by queued work on any stream of this device
        cudaDeviceSynchronize();
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t nb = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&b.p, nb);
    if (e != cudaSuccess) {
        b.p = nullptr;
        set_error("cudaMalloc(%zu) failed: %s", nb, cudaGetErrorString(e));
        return SOAP_ENOMEM;
    }
    b.bytes = nb;
    return SOAP_OK;
}

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

soap_status ensure_host(HostBuf& b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return SOAP_OK;
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMallocHost(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        set_error("cudaMallocHost(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return SOAP_ENOMEM;
    }
    b.bytes = bytes;
    return SOAP_OK;
}

void release_host(HostBuf& b) {
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// Device-side copy of n bytes from mapped pinned host memory (the ring) into device memory.
// A kernel, not a copy-engine transfer: a small upload on the compute stream must not queue
// behind a large upload that the copy engine is running for the upload stream.
__global__ void k_ring_fetch(const unsigned char* __restrict__ src, unsigned char* __restrict__ dst,
                             size_t n) {
    const size_t n8 = n / 8;
    const uint64_t* s8 = reinterpret_cast<const uint64_t*>(src);
    uint64_t* d8 = reinterpret_cast<uint64_t*>(dst);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n8; i += (size_t)gridDim.x * blockDim.x)
        d8[i] = s8[i];
    if (blockIdx.x == 0 && threadIdx.x < n - n8 * 8) dst[n8 * 8 + threadIdx.x] = src[n8 * 8 + threadIdx.x];
}

soap_status upload_small(soap_ctx* c, void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return SOAP_OK;
    PinnedRing& R = c->ring;
    const size_t need = (bytes + 255) / 256 * 256;
    if (need > kRingBytes / 4) {                       // large: a plain (pageable) copy
        SOAP_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
        return SOAP_OK;
    }
    if (!R.p) {
        void* h = nullptr;
        cudaError_t e = cudaMallocHost(&h, kRingBytes);
        if (e != cudaSuccess) {
            set_error("cudaMallocHost(%zu) failed: %s", kRingBytes, cudaGetErrorString(e));
            return SOAP_ENOMEM;
        }
        R.p = static_cast<unsigned char*>(h);
        R.cap = kRingBytes;
        R.head = 0;
        void* dp = nullptr;
        SOAP_CUDA(cudaHostGetDevicePointer(&dp, h, 0));
        R.dev = static_cast<unsigned char*>(dp);
    }
    if (R.head + need > R.cap) R.head = 0;
    const size_t lo = R.head, hi = R.head + need;
    // the oldest uses are the ones in the way: wait for those that overlap [lo, hi)
    size_t done = 0;
    while (done < R.pending.size() && R.pending[done].lo < hi && R.pending[done].hi > lo) {
        SOAP_CUDA(cudaEventSynchronize(R.pending[done].ev));
        R.free_ev.push_back(R.pending[done].ev);
        done++;
    }
    R.pending.erase(R.pending.begin(), R.pending.begin() + (long)done);
    std::memcpy(R.p + lo, src, bytes);
    const bool aligned = (reinterpret_cast<uintptr_t>(dst) % 8) == 0;
    if (aligned) {
        const size_t n8 = bytes / 8;
        const unsigned grid = (unsigned)std::min<size_t>((n8 + 255) / 256 + 1, 152 * 4);
        k_ring_fetch<<<grid, 256, 0, c->stream>>>(R.dev + lo, static_cast<unsigned char*>(dst), bytes);
        SOAP_CUDA(cudaGetLastError());
        SOAP_LAUNCHED(c);
    } else {
        SOAP_CUDA(cudaMemcpyAsync(dst, R.p + lo, bytes, cudaMemcpyHostToDevice, c->stream));
    }
    cudaEvent_t ev = nullptr;
    if (!R.free_ev.empty()) {
        ev = R.free_ev.back();
        R.free_ev.pop_back();
    } else {
        SOAP_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    SOAP_CUDA(cudaEventRecord(ev, c->stream));
    R.pending.push_back({lo, hi, ev});
    R.head = hi;
    return SOAP_OK;
}

void ring_release(soap_ctx* c) {
    PinnedRing& R = c->ring;
    for (auto& u : R.pending) {
        cudaEventSynchronize(u.ev);
        cudaEventDestroy(u.ev);
    }
    for (cudaEvent_t e : R.free_ev) cudaEventDestroy(e);
    R.pending.clear();
    R.free_ev.clear();
    if (R.p) cudaFreeHost(R.p);
    R.p = nullptr;
    R.dev = nullptr;
    R.cap = R.head = 0;
}

static bool is_finite(double x) { return std::isfinite(x); }

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Copy n bytes of a caller array into device memory `dst` (async on the context stream).
static soap_status to_device(soap_ctx* c, void* dst, const void* src, size_t n, int on_device) {
    SOAP_CUDA(cudaMemcpyAsync(dst, src, n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
    return SOAP_OK;
}

// Streams and events of the host-transfer pipeline, created on first use.
static soap_status ensure_pipeline(soap_ctx* c) {
    if (c->in_stream) return SOAP_OK;
    SOAP_CUDA(cudaStreamCreateWithFlags(&c->in_stream, cudaStreamNonBlocking));
    SOAP_CUDA(cudaStreamCreateWithFlags(&c->out_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 3; i++) {
        SOAP_CUDA(cudaEventCreateWithFlags(&c->up_filled[i], cudaEventDisableTiming));
        SOAP_CUDA(cudaEventCreateWithFlags(&c->up_free[i], cudaEventDisableTiming));
    }
    for (int i = 0; i < 2; i++) {
        SOAP_CUDA(cudaEventCreateWithFlags(&c->dn_spec[i], cudaEventDisableTiming));
        SOAP_CUDA(cudaEventCreateWithFlags(&c->dn_rv[i], cudaEventDisableTiming));
        SOAP_CUDA(cudaEventCreateWithFlags(&c->dn_free[i], cudaEventDisableTiming));
    }
    return SOAP_OK;
}

static void sync_all(soap_ctx* c) {
    if (c->in_stream) cudaStreamSynchronize(c->in_stream);
    join_geometry(c);
    if (c->aux2) cudaStreamSynchronize(c->aux2);
    if (c->aux) cudaStreamSynchronize(c->aux);
    cudaStreamSynchronize(c->stream);
    if (c->out_stream) cudaStreamSynchronize(c->out_stream);
}

static void destroy_pipeline(soap_ctx* c) {
    if (!c->in_stream) return;
    sync_all(c);
    for (int i = 0; i < 3; i++) {
        cudaEventDestroy(c->up_filled[i]);
        cudaEventDestroy(c->up_free[i]);
        release(c->up_stage[i]);
    }
    for (int i = 0; i < 2; i++) {
        cudaEventDestroy(c->dn_spec[i]);
        cudaEventDestroy(c->dn_rv[i]);
        cudaEventDestroy(c->dn_free[i]);
        release(c->dn_stage[i]);
    }
    cudaStreamDestroy(c->in_stream);
    cudaStreamDestroy(c->out_stream);
    c->in_stream = c->out_stream = nullptr;
}

static void free_ctx_memory(soap_ctx* c) {
    void* ptrs[] = {c->cell_I, c->cell_w, c->cell_mu, c->cell_j, c->cell_bin, c->cell_mu32,
                    c->cell_k0, c->cell_k1, c->flags, c->q64,
                    c->q32, c->a64[0], c->a32[0], c->a64[1], c->a32[1], c->kq_fixed,
                    c->sum_I_fixed, c->qtoff, c->qgstart, c->qc64, c->qc32, c->geo_counter, c->cell_x,
                    c->qgrp, c->qgrp_start};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    DevBuf* bufs[] = {&c->stage_in, &c->fq, &c->contrast, &c->kphase, &c->jobs, &c->coefs, &c->job_counters,
                      &c->regions, &c->region_geo, &c->phases, &c->out_stage, &c->partial, &c->ccf.tmp,
                      &c->ccf.tab, &c->lsf_taps, &c->lsf_tmp, &c->bis_tab, &c->tc_coef, &c->ccf.m,
                      &c->tm_planes, &c->tm_coef, &c->dir_cells, &c->dir_count, &c->dir_rows};
    for (DevBuf* b : bufs) release(*b);
    release_host(c->host_stage);
    ring_release(c);
    for (cudaStream_t* s : {&c->aux, &c->aux2})
        if (*s) {
            cudaStreamSynchronize(*s);
            cudaStreamDestroy(*s);
            *s = nullptr;
        }
    for (cudaEvent_t* e : {&c->ev_fork, &c->ev_geo, &c->ev_rg, &c->ev_ph, &c->ev_main})
        if (*e) { cudaEventDestroy(*e); *e = nullptr; }
}

// upload [n_mu][n_px] local spectra into padded rows: float64 sources fill the fp64 and fp32
// rows, float32 sources (f32src) the fp32 rows only.  With the host-transfer pipeline on, a
// host source is copied on in_stream into its own stage (slot: 0 quiet, 1 spot, 2 facula) and
// the compute stream waits for that copy only.
static soap_status upload_spectra(soap_ctx* c, const void* src, int on_device, int f32src,
                                  double* dst64, float* dst32, int slot) {
    size_t bytes = (size_t)c->n_mu * (size_t)c->n_px * (f32src ? sizeof(float) : sizeof(double));
    const void* dsrc = src;
    if (!on_device && c->host_async) {
        SOAP_TRY(ensure_pipeline(c));
        soap::DevBuf& st = c->up_stage[slot];
        SOAP_TRY(ensure(st, bytes));
        SOAP_CUDA(cudaStreamWaitEvent(c->in_stream, c->up_free[slot], 0));   // last read of the stage
        SOAP_CUDA(cudaMemcpyAsync(st.p, src, bytes, cudaMemcpyHostToDevice, c->in_stream));
        SOAP_CUDA(cudaEventRecord(c->up_filled[slot], c->in_stream));
        SOAP_CUDA(cudaStreamWaitEvent(c->stream, c->up_filled[slot], 0));
        dsrc = st.p;
    } else if (!on_device) {
        SOAP_TRY(ensure(c->stage_in, bytes));
        SOAP_TRY(to_device(c, c->stage_in.p, src, bytes, 0));
        dsrc = c->stage_in.p;
    }
    if (f32src) SOAP_TRY(pad_rows32(c, static_cast<const float*>(dsrc), dst32, c->n_mu));
    else SOAP_TRY(pad_rows(c, static_cast<const double*>(dsrc), dst64, dst32, c->n_mu));
    c->rows_version++;                      // derived copies of the rows (BF16 planes) are stale
    if (!on_device && c->host_async) SOAP_CUDA(cudaEventRecord(c->up_free[slot], c->stream));
    return SOAP_OK;
}

// Sets bits in the device status word as a failing kernel would (soap_debug_inject_timeout).
__global__ void k_raise_status(unsigned int* flags, unsigned int bits) { atomicOr(flags, bits); }

static soap_status check_flags(soap_ctx* c) {
    unsigned int f = 0;
    SOAP_TRY(join_geometry(c));
    SOAP_CUDA(cudaMemcpyAsync(&f, c->flags, sizeof(f), cudaMemcpyDeviceToHost, c->stream));
    SOAP_CUDA(cudaStreamSynchronize(c->stream));
    if (f) {
        cudaMemsetAsync(c->flags, 0, sizeof(unsigned int), c->stream);
        set_error("device status word 0x%x (tap range %d, box range %d, job overflow %d, bisector order %d, "
                  "tensor-core wait timeout %d)", f, !!(f & kFlagTapRange), !!(f & kFlagBoxRange),
                  !!(f & kFlagJobOverflow), !!(f & kFlagOrder), !!(f & kFlagTimeout));
        return (f & kFlagTimeout) ? SOAP_ETIMEOUT : SOAP_ERANGE;
    }
    return SOAP_OK;
}

cudaEvent_t timer_begin(soap_ctx* c) {
    cudaEvent_t e = nullptr;
    if (!c->event_pool.empty()) {
        e = c->event_pool.back();
        c->event_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return nullptr;
    }
    cudaEventRecord(e, c->stream);
    return e;
}

void timer_end(soap_ctx* c, int timer, cudaEvent_t begin) {
    if (!begin) return;
    cudaEvent_t e = nullptr;
    if (!c->event_pool.empty()) {
        e = c->event_pool.back();
        c->event_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        c->event_pool.push_back(begin);
        return;
    }
    cudaEventRecord(e, c->stream);
    c->pending.push_back({timer, begin, e});
}

static soap_status fold_timers(soap_ctx* c) {
    if (c->pending.empty()) return SOAP_OK;
    SOAP_CUDA(cudaStreamSynchronize(c->stream));
    if (c->aux2) SOAP_CUDA(cudaStreamSynchronize(c->aux2));
    if (c->aux) SOAP_CUDA(cudaStreamSynchronize(c->aux));
    for (auto& t : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            c->timer_ms[t.timer] += ms;
            c->timer_n[t.timer] += 1;
        }
        c->event_pool.push_back(t.a);
        c->event_pool.push_back(t.b);
    }
    c->pending.clear();
    return SOAP_OK;
}

static void destroy_events(soap_ctx* c) {
    for (auto& t : c->pending) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    c->pending.clear();
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    c->event_pool.clear();
}

// Validate a star description; fills delta and the tap range.
static soap_status check_star(const soap_star_desc* s, double* delta_out, int64_t* tmin_out,
                              int64_t* tmax_out) {
    if (!s) { set_error("star is NULL"); return SOAP_EINVAL; }
    if (s->grid_n < 1 || s->grid_n > 8192) { set_error("grid_n=%d outside 1..8192", s->grid_n); return SOAP_EINVAL; }
    if (s->n_mu < 1 || s->n_mu > SOAP_MAX_MU) { set_error("n_mu=%d outside 1..%d", s->n_mu, SOAP_MAX_MU); return SOAP_ERANGE; }
    if (s->n_px < 2 || s->n_px > (int64_t(1) << 28)) { set_error("n_px=%lld outside 2..2^28", (long long)s->n_px); return SOAP_EINVAL; }
    double vals[] = {s->vsini_kms, s->incl_deg, s->u1, s->u2, s->diff_rot_alpha,
                     s->lambda_start_A, s->lambda_end_A, s->t_quiet_K};
    for (double v : vals)
        if (!is_finite(v)) { set_error("non-finite star parameter"); return SOAP_EINVAL; }
    if (!(s->lambda_start_A > 0) || !(s->lambda_end_A > s->lambda_start_A)) {
        set_error("need 0 < lambda_start < lambda_end"); return SOAP_EINVAL;
    }
    if (s->incl_deg < 0 || s->incl_deg > 180) { set_error("incl_deg outside [0,180]"); return SOAP_EINVAL; }
    if (!(s->t_quiet_K > 0)) { set_error("t_quiet_K must be > 0"); return SOAP_EINVAL; }
    if (!s->mu_values) { set_error("mu_values is NULL"); return SOAP_EINVAL; }
    for (int b = 0; b < s->n_mu; b++)
        if (!is_finite(s->mu_values[b]) || !(s->mu_values[b] > 0) || s->mu_values[b] > 1) {
            set_error("mu_values[%d] outside (0,1]", b); return SOAP_EINVAL;
        }
    double vfac = std::fmax(1.0, std::fabs(1.0 + s->diff_rot_alpha));
    double vmax = std::fabs(s->vsini_kms) * vfac;
    if (!(vmax < kCKms)) { set_error("|v| >= c"); return SOAP_EINVAL; }
    double delta = std::log1p((s->lambda_end_A - s->lambda_start_A) / s->lambda_start_A) / (double)(s->n_px - 1);
    if (!(delta > 0) || !is_finite(delta)) { set_error("grid step Delta not positive"); return SOAP_EINVAL; }
    double smax = std::atanh(vmax / kCKms) / delta;
    if (!(smax < 1e6)) { set_error("velocity shift too large for the pixel size"); return SOAP_ERANGE; }
    int64_t tmax = (int64_t)std::ceil(smax) + 1, tmin = (int64_t)std::floor(-smax) - 1;
    if (tmax - tmin + 1 > SOAP_MAX_TAPS) {
        set_error("velocity kernel needs %lld taps > %d (vsini too large for the pixel size)",
                  (long long)(tmax - tmin + 1), SOAP_MAX_TAPS);
        return SOAP_ERANGE;
    }
    *delta_out = delta;
    *tmin_out = tmin;
    *tmax_out = tmax;
    return SOAP_OK;
}

static void set_star_params(soap_ctx* c, const soap_star_desc* s) {
    c->vsini = s->vsini_kms; c->incl_deg = s->incl_deg; c->u1 = s->u1; c->u2 = s->u2;
    c->alpha = s->diff_rot_alpha; c->t_quiet = s->t_quiet_K;
    for (int b = 0; b < s->n_mu; b++) c->mu_values[b] = s->mu_values[b];
    c->mu_sorted = 1;
    for (int b = 1; b < s->n_mu; b++)
        if (!(s->mu_values[b] - s->mu_values[b - 1] > 1e-9)) c->mu_sorted = 0;
    // fixed-point kernels: every partial sum is bounded by sum |I| <= 4 (1 + |u1| + |u2|)
    double bound = 4.0 * (1.0 + std::fabs(s->u1) + std::fabs(s->u2));
    c->fx_bits = 61 - (int)std::ceil(std::log2(bound));
}

}  // namespace soap

using namespace soap;

extern "C" {

const char* soap_last_error(void) { return g_error; }

soap_status soap_init_star(const soap_star_desc* s, const double* quiet_local, int quiet_on_device,
                           void* cuda_stream, soap_ctx** out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return SOAP_EINVAL; }
    *out = nullptr;
    if (!s || !quiet_local) { set_error("star or quiet_local is NULL"); return SOAP_EINVAL; }
    double delta = 0;
    int64_t tmin = 0, tmax = 0;
    SOAP_TRY(check_star(s, &delta, &tmin, &tmax));

    soap_ctx* c = new (std::nothrow) soap_ctx();
    if (!c) { set_error("out of host memory"); return SOAP_ENOMEM; }
    cudaGetDevice(&c->device);
    c->stream = (cudaStream_t)cuda_stream;
    c->N = s->grid_n; c->n_mu = s->n_mu; c->n_px = s->n_px;
    c->lam_s = s->lambda_start_A; c->lam_e = s->lambda_end_A; c->delta = delta;
    set_star_params(c, s);
    c->tap_min = (int)tmin;
    c->n_taps = (int)(tmax - tmin + 1);
    int64_t need = std::max<int64_t>(tmax, -tmin) + 1;
    // 32 more than the taps need: the direct form reads 16-byte vectors up to 20 values past a
    // pixel and rounds its start down to a vector boundary
    c->pad = round_up(need + 32, 32);
    // rows reach past the last tile of any contraction (tiles of up to 1024 pixels)
    c->row_len = round_up(round_up(c->n_px, 1024) + 2 * c->pad, 32);

    soap_status st = SOAP_OK;
    size_t NN = (size_t)c->N * c->N;
    size_t rows = (size_t)c->n_mu * (size_t)c->row_len;
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes) if (e == cudaSuccess) e = cudaMalloc((void**)&(ptr), (bytes))
    ALLOC(c->cell_I, NN * sizeof(double));
    ALLOC(c->cell_w, NN * sizeof(double));
    ALLOC(c->cell_mu, NN * sizeof(double));
    ALLOC(c->cell_j, NN * sizeof(int32_t));
    ALLOC(c->cell_bin, NN * sizeof(int32_t));
    ALLOC(c->cell_mu32, NN * sizeof(float));
    ALLOC(c->cell_k0, NN * sizeof(long long));
    ALLOC(c->cell_k1, NN * sizeof(long long));
    ALLOC(c->flags, sizeof(unsigned int));
    ALLOC(c->q64, rows * sizeof(double));
    ALLOC(c->q32, rows * sizeof(float));
    ALLOC(c->kq_fixed, (size_t)c->n_mu * SOAP_MAX_TAPS * sizeof(long long));
    ALLOC(c->sum_I_fixed, 2 * sizeof(long long));
    ALLOC(c->qtoff, (size_t)c->n_mu * SOAP_MAX_TAPS * sizeof(long long));
    ALLOC(c->qgstart, 2 * sizeof(int));
    ALLOC(c->qgrp, (size_t)c->n_mu * (SOAP_MAX_TAPS + 1) * sizeof(soap::TapGroup));
    ALLOC(c->qgrp_start, 2 * sizeof(int));
    ALLOC(c->qc64, (size_t)c->n_mu * SOAP_MAX_TAPS * sizeof(double));
    ALLOC(c->qc32, (size_t)c->n_mu * SOAP_MAX_TAPS * sizeof(float));
    ALLOC(c->geo_counter, sizeof(int));
    ALLOC(c->cell_x, (size_t)c->N * sizeof(double));
#undef ALLOC
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux2, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&c->ev_fork, &c->ev_geo, &c->ev_rg, &c->ev_ph, &c->ev_main})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        set_error("device allocation failed: %s", cudaGetErrorString(e));
        free_ctx_memory(c);
        delete c;
        return SOAP_ENOMEM;
    }
    st = SOAP_OK;
    if (cudaMemsetAsync(c->flags, 0, sizeof(unsigned int), c->stream) != cudaSuccess) st = SOAP_ECUDA;
    {
        // cell centres (2 i + 1 - N) / N, IEEE-divided here once instead of in every cell
        std::vector<double> xs((size_t)c->N);
        for (int i = 0; i < c->N; i++) xs[(size_t)i] = (double)(2 * i + 1 - c->N) / (double)c->N;
        if (st == SOAP_OK &&
            cudaMemcpy(c->cell_x, xs.data(), xs.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            st = SOAP_ECUDA;
    }
    if (st == SOAP_OK) st = geometry_init(c);
    if (st == SOAP_OK) st = upload_spectra(c, quiet_local, quiet_on_device, 0, c->q64, c->q32, 0);
    c->q64_ok = st == SOAP_OK;
    if (st == SOAP_OK) st = check_flags(c);
    if (st != SOAP_OK) {
        cudaStreamSynchronize(c->stream);
        free_ctx_memory(c);
        delete c;
        return st;
    }
    *out = c;
    return SOAP_OK;
}

soap_status soap_update_star(soap_ctx* c, const soap_star_desc* s) {
    clear_error();
    if (!c || !s) { set_error("ctx or star is NULL"); return SOAP_EINVAL; }
    double delta = 0;
    int64_t tmin = 0, tmax = 0;
    SOAP_TRY(check_star(s, &delta, &tmin, &tmax));
    if (s->grid_n != c->N || s->n_mu != c->n_mu || s->n_px != c->n_px ||
        s->lambda_start_A != c->lam_s || s->lambda_end_A != c->lam_e) {
        set_error("soap_update_star cannot change grid_n, n_mu, n_px or the wavelength range");
        return SOAP_EINVAL;
    }
    if (std::max<int64_t>(tmax, -tmin) + 1 > c->pad) {
        set_error("the new velocity kernels need more row padding than this context has");
        return SOAP_ERANGE;
    }
    set_star_params(c, s);
    c->tap_min = (int)tmin;
    c->n_taps = (int)(tmax - tmin + 1);
    return geometry_init(c);
}

soap_status soap_set_quiet_spectrum(soap_ctx* c, const double* quiet_local, int on_device) {
    clear_error();
    if (!c || !quiet_local) { set_error("ctx or quiet_local is NULL"); return SOAP_EINVAL; }
    SOAP_TRY(upload_spectra(c, quiet_local, on_device, 0, c->q64, c->q32, 0));
    c->q64_ok = true;
    return SOAP_OK;
}

soap_status soap_set_quiet_spectrum_f32(soap_ctx* c, const float* quiet_local, int on_device) {
    clear_error();
    if (!c || !quiet_local) { set_error("ctx or quiet_local is NULL"); return SOAP_EINVAL; }
    c->q64_ok = false;
    return upload_spectra(c, quiet_local, on_device, 1, nullptr, c->q32, 0);
}

soap_status soap_set_profiling(soap_ctx* c, int enabled) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return SOAP_EINVAL; }
    c->profiling = enabled != 0;
    return SOAP_OK;
}

soap_status soap_get_kernel_time(soap_ctx* c, int32_t timer, double* total_ms, uint64_t* launches) {
    clear_error();
    if (!c || !total_ms || !launches) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (timer < 0 || timer >= SOAP_TIMER_COUNT) { set_error("unknown timer %d", timer); return SOAP_EINVAL; }
    SOAP_TRY(fold_timers(c));
    *total_ms = c->timer_ms[timer];
    *launches = c->timer_n[timer];
    return SOAP_OK;
}

soap_status soap_reset_kernel_times(soap_ctx* c) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return SOAP_EINVAL; }
    SOAP_TRY(fold_timers(c));
    for (int k = 0; k < SOAP_TIMER_COUNT; k++) { c->timer_ms[k] = 0; c->timer_n[k] = 0; }
    return SOAP_OK;
}

static soap_status set_active(soap_ctx* c, int32_t type, const void* active_local, int on_device,
                              int f32src) {
    if (!c || !active_local) { set_error("ctx or active_local is NULL"); return SOAP_EINVAL; }
    if (type != SOAP_SPOT && type != SOAP_FACULA) { set_error("type must be SOAP_SPOT or SOAP_FACULA"); return SOAP_EINVAL; }
    int t = type - 1;
    size_t rows = (size_t)c->n_mu * (size_t)c->row_len;
    if (!c->a64[t]) {
        if (cudaMalloc((void**)&c->a64[t], rows * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void**)&c->a32[t], rows * sizeof(float)) != cudaSuccess) {
            set_error("device allocation of active spectra failed");
            return SOAP_ENOMEM;
        }
    }
    c->a64_ok[t] = false;
    SOAP_TRY(upload_spectra(c, active_local, on_device, f32src, c->a64[t], c->a32[t], 1 + t));
    c->active_set[t] = true;
    c->a64_ok[t] = !f32src;
    return SOAP_OK;
}

soap_status soap_set_active_spectrum(soap_ctx* c, int32_t type, const double* active_local,
                                     int on_device) {
    clear_error();
    return set_active(c, type, active_local, on_device, 0);
}

soap_status soap_set_active_spectrum_f32(soap_ctx* c, int32_t type, const float* active_local,
                                         int on_device) {
    clear_error();
    return set_active(c, type, active_local, on_device, 1);
}

soap_status soap_set_stream(soap_ctx* c, void* stream) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return SOAP_EINVAL; }
    c->stream = (cudaStream_t)stream;
    return SOAP_OK;
}

soap_status soap_synchronize(soap_ctx* c) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return SOAP_EINVAL; }
    if (c->in_stream) SOAP_CUDA(cudaStreamSynchronize(c->in_stream));
    SOAP_TRY(check_flags(c));
    if (c->out_stream) SOAP_CUDA(cudaStreamSynchronize(c->out_stream));
    return SOAP_OK;
}

soap_status soap_set_facula_limb_brightening(soap_ctx* c, int enabled) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return SOAP_EINVAL; }
    c->facula_mu = enabled != 0;
    return SOAP_OK;
}

soap_status soap_set_ccf_tensor_cores(soap_ctx* c, int enabled) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return SOAP_EINVAL; }
    c->ccf_tc = enabled != 0;
    return SOAP_OK;
}

soap_status soap_set_host_async(soap_ctx* c, int enabled) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return SOAP_EINVAL; }
    if (enabled) {
        SOAP_TRY(ensure_pipeline(c));
    } else if (c->host_async) {
        sync_all(c);
    }
    c->host_async = enabled != 0;
    return SOAP_OK;
}

soap_status soap_get_star_info(soap_ctx* c, soap_star_info* out) {
    clear_error();
    if (!c || !out) { set_error("ctx or out is NULL"); return SOAP_EINVAL; }
    long long h2[2] = {0, 0};
    SOAP_TRY(join_geometry(c));
    SOAP_CUDA(cudaMemcpyAsync(h2, c->sum_I_fixed, sizeof(h2), cudaMemcpyDeviceToHost, c->stream));
    SOAP_TRY(check_flags(c));
    c->total_I = std::ldexp((double)h2[0], -c->fx_bits);
    c->n_visible = h2[1];
    memset(out, 0, sizeof(*out));
    out->n_visible = c->n_visible;
    out->tap_min = c->tap_min;
    out->n_taps = c->n_taps;
    out->delta = c->delta;
    out->total_intensity = c->total_I;
    out->fixed_point_bits = c->fx_bits;
    return SOAP_OK;
}

soap_status soap_get_launch_count(const soap_ctx* c, uint64_t* out) {
    clear_error();
    if (!c || !out) { set_error("ctx or out is NULL"); return SOAP_EINVAL; }
    *out = c->launches;
    return SOAP_OK;
}

soap_status soap_debug_inject_timeout(soap_ctx* c) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return SOAP_EINVAL; }
    k_raise_status<<<1, 1, 0, c->stream>>>(c->flags, kFlagTimeout);
    SOAP_CUDA(cudaGetLastError());
    return SOAP_OK;
}

soap_status soap_quiet_spectrum(soap_ctx* c, int32_t form, int32_t precision, void* out,
                                int out_on_device) {
    clear_error();
    if (!c || !out) { set_error("ctx or out is NULL"); return SOAP_EINVAL; }
    if (form != SOAP_FORM_TOEPLITZ && form != SOAP_FORM_DIRECT) { set_error("unknown form %d", form); return SOAP_EINVAL; }
    if (precision != SOAP_FP64 && precision != SOAP_FP32) { set_error("unknown precision %d", precision); return SOAP_EINVAL; }
    if (precision == SOAP_FP64 && !c->q64_ok) {
        set_error("the FP64 path needs float64 local spectra (the quiet ones were set in float32)");
        return SOAP_ESTATE;
    }
    size_t esz = precision == SOAP_FP64 ? 8 : 4;
    size_t bytes = (size_t)c->n_px * esz;
    void* dst = out;
    if (!out_on_device) {
        SOAP_TRY(ensure(c->out_stage, bytes));
        dst = c->out_stage.p;
    }
    void* raw = dst;                               // before the instrument's line-spread function
    if (c->lsf_K >= 0) {
        SOAP_TRY(ensure(c->lsf_tmp, bytes));
        raw = c->lsf_tmp.p;
    }
    if (form == SOAP_FORM_TOEPLITZ) SOAP_TRY(toeplitz_quiet(c, precision, raw));
    else SOAP_TRY(direct_quiet(c, precision, raw));
    if (c->lsf_K >= 0) SOAP_TRY(launch_lsf(c, raw, dst, precision == SOAP_FP32, 1));
    if (!out_on_device) {
        SOAP_CUDA(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
        SOAP_CUDA(cudaStreamSynchronize(c->stream));
    }
    return SOAP_OK;
}

}  // extern "C"

// Checks of soap_active_phases / soap_active_rv arguments; the regions in device form and
// their (type, temperature) classes.
struct ActiveArgs {
    std::vector<RegionDev> rd;
    double ctemp[SOAP_MAX_CLASSES];
    int ctype[SOAP_MAX_CLASSES];
    int n_class = 0;
};

static soap_status check_active(soap_ctx* c, const soap_region* regions, int32_t n_regions,
                                const double* phases, int32_t n_phases, uint32_t effects,
                                int32_t precision, ActiveArgs& A) {
    if (n_regions < 0 || n_regions > SOAP_MAX_REGIONS) { set_error("n_regions=%d outside 0..%d", n_regions, SOAP_MAX_REGIONS); return SOAP_ERANGE; }
    if (n_regions > 0 && !regions) { set_error("regions is NULL"); return SOAP_EINVAL; }
    if (n_phases < 0) { set_error("n_phases < 0"); return SOAP_EINVAL; }
    if (n_phases > 0 && !phases) { set_error("phases is NULL"); return SOAP_EINVAL; }
    if (effects == 0 || (effects & ~7u)) { set_error("effects must be a non-empty OR of SOAP_EFFECT_*"); return SOAP_EINVAL; }
    if (precision != SOAP_FP64 && precision != SOAP_FP32 && precision != SOAP_BF16X3) {
        set_error("unknown precision %d", precision);
        return SOAP_EINVAL;
    }
    for (int p = 0; p < n_phases; p++)
        if (!is_finite(phases[p])) { set_error("phases[%d] not finite", p); return SOAP_EINVAL; }
    A.rd.resize(n_regions);
    A.n_class = 0;
    for (int r = 0; r < n_regions; r++) {
        const soap_region& g = regions[r];
        if (g.type != SOAP_SPOT && g.type != SOAP_FACULA) { set_error("regions[%d].type invalid", r); return SOAP_EINVAL; }
        if (g.reserved != 0) { set_error("regions[%d].reserved must be 0", r); return SOAP_EINVAL; }
        if (!is_finite(g.lat_deg) || !is_finite(g.lon_deg) || !is_finite(g.radius_rstar) || !is_finite(g.temp_K)) {
            set_error("regions[%d] has a non-finite field", r); return SOAP_EINVAL;
        }
        if (g.radius_rstar < 0 || g.radius_rstar > 1) { set_error("regions[%d].radius_rstar outside [0,1]", r); return SOAP_EINVAL; }
        if (!(g.temp_K > 0)) { set_error("regions[%d].temp_K must be > 0", r); return SOAP_EINVAL; }
        int cl = -1;
        for (int k = 0; k < A.n_class; k++)
            if (A.ctype[k] == g.type && A.ctemp[k] == g.temp_K) cl = k;
        if (cl < 0) {
            if (A.n_class == SOAP_MAX_CLASSES) { set_error("more than %d distinct (type, temperature) pairs", SOAP_MAX_CLASSES); return SOAP_ERANGE; }
            cl = A.n_class++;
            A.ctype[cl] = g.type;
            A.ctemp[cl] = g.temp_K;
        }
        A.rd[r] = RegionDev{g.lat_deg, g.lon_deg, g.radius_rstar, g.temp_K, g.type, cl};
    }
    for (int k = 0; k < A.n_class; k++) {
        bool ok = A.ctype[k] == SOAP_SPOT ? c->active_set[0] : (c->active_set[1] || c->active_set[0]);
        if (!ok) { set_error("no active spectrum set for region type %d", A.ctype[k]); return SOAP_ESTATE; }
    }
    if (precision == SOAP_FP64 && (!c->q64_ok || (c->active_set[0] && !c->a64_ok[0]) ||
                                   (c->active_set[1] && !c->a64_ok[1]))) {
        set_error("the FP64 path needs float64 local spectra (some were set in float32)");
        return SOAP_ESTATE;
    }
    return SOAP_OK;
}

// Checks of the CCF / RV arguments (soap_rv_ccf, soap_active_rv).
static soap_status check_rv(soap_ctx* c, const double* mask_lambda, const double* mask_weight,
                            int32_t n_lines, double mask_width_kms, double v_lo, double v_step,
                            int32_t n_v) {
    if (!mask_lambda || !mask_weight) { set_error("NULL mask"); return SOAP_EINVAL; }
    if (n_lines < 1 || n_v < 5 || n_v > 4096) { set_error("need n_lines >= 1, 5 <= n_v <= 4096"); return SOAP_EINVAL; }
    if (!is_finite(mask_width_kms) || !(mask_width_kms > 0) || !is_finite(v_lo) || !is_finite(v_step) || !(v_step > 0)) {
        set_error("mask width / velocity grid invalid"); return SOAP_EINVAL;
    }
    double v_hi = v_lo + v_step * (n_v - 1);
    if (!(std::fabs(v_lo) < kCKms) || !(std::fabs(v_hi) < kCKms)) { set_error("velocity grid reaches c"); return SOAP_EINVAL; }
    double h = mask_width_kms / (2.0 * kCKms * c->delta);
    if (2.0 * h > 14.0) { set_error("mask box spans more than 14 pixels"); return SOAP_ERANGE; }
    if (ccf_mask_same(c->ccf, mask_lambda, mask_weight, n_lines, mask_width_kms)) return SOAP_OK;   // checked before
    for (int l = 0; l < n_lines; l++)
        if (!is_finite(mask_lambda[l]) || !(mask_lambda[l] > 0) || !is_finite(mask_weight[l])) {
            set_error("mask line %d invalid", l); return SOAP_EINVAL;
        }
    return SOAP_OK;
}

// Spectra of one effect into dst, through the instrument's line-spread function when one is set.
static soap_status active_lsf(soap_ctx* c, const ActiveArgs& A, int32_t n_regions, const double* phases,
                              int32_t n_phases, uint32_t effect, int32_t precision, void* dst, size_t bytes) {
    void* raw = dst;
    if (c->lsf_K >= 0) {
        SOAP_TRY(ensure(c->lsf_tmp, bytes));
        raw = c->lsf_tmp.p;
    }
    SOAP_TRY(toeplitz_active(c, A.rd.data(), n_regions, A.ctemp, A.ctype, A.n_class, phases, n_phases,
                             effect, precision, raw));
    if (c->lsf_K >= 0) SOAP_TRY(launch_lsf(c, raw, dst, precision != SOAP_FP64, n_phases));
    return SOAP_OK;
}

extern "C" {

soap_status soap_set_instrument_resolution(soap_ctx* c, double resolving_power) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return SOAP_EINVAL; }
    if (!(resolving_power >= 0) || !std::isfinite(resolving_power)) {
        set_error("resolving power must be finite and >= 0 (0: off)"); return SOAP_EINVAL;
    }
    return set_instrument(c, resolving_power);
}

soap_status soap_inject_bisectors(soap_ctx* c, const double* in, double* out, int32_t n_rows,
                                  const double* bis_table, const double* orig_table, int32_t n_depth,
                                  int on_device) {
    clear_error();
    if (!c || !in || !out || !bis_table || !orig_table) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (n_rows < 0 || n_depth < 2) { set_error("need n_rows >= 0 and n_depth >= 2"); return SOAP_EINVAL; }
    if (in == out) { set_error("in and out must not be the same array"); return SOAP_EINVAL; }
    if (n_rows == 0) return SOAP_OK;
    const size_t bytes = (size_t)n_rows * (size_t)c->n_px * sizeof(double);
    const double* din = in;
    double* dout = out;
    if (!on_device) {
        SOAP_TRY(ensure(c->lsf_tmp, bytes));
        SOAP_TRY(ensure(c->out_stage, bytes));
        SOAP_CUDA(cudaMemcpyAsync(c->lsf_tmp.p, in, bytes, cudaMemcpyHostToDevice, c->stream));
        din = c->lsf_tmp.as<double>();
        dout = c->out_stage.as<double>();
    }
    SOAP_TRY(inject_bisectors(c, din, dout, n_rows, bis_table, orig_table, n_depth));
    if (!on_device) SOAP_CUDA(cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, c->stream));
    return check_flags(c);
}

soap_status soap_lower_resolution(soap_ctx* c, const void* in, void* out, int32_t spectra_f32,
                                  int32_t n_spec, int on_device) {
    clear_error();
    if (!c || !in || !out) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (c->lsf_K < 0) { set_error("no instrument resolution set (soap_set_instrument_resolution)"); return SOAP_ESTATE; }
    if (n_spec < 0) { set_error("n_spec < 0"); return SOAP_EINVAL; }
    if (in == out) { set_error("in and out must not be the same array"); return SOAP_EINVAL; }
    if (n_spec == 0) return SOAP_OK;
    const size_t bytes = (size_t)n_spec * (size_t)c->n_px * (spectra_f32 ? 4 : 8);
    if (on_device) return launch_lsf(c, in, out, spectra_f32 ? 1 : 0, n_spec);
    SOAP_TRY(ensure(c->lsf_tmp, bytes));
    SOAP_TRY(ensure(c->out_stage, bytes));
    SOAP_CUDA(cudaMemcpyAsync(c->lsf_tmp.p, in, bytes, cudaMemcpyHostToDevice, c->stream));
    SOAP_TRY(launch_lsf(c, c->lsf_tmp.p, c->out_stage.p, spectra_f32 ? 1 : 0, n_spec));
    SOAP_CUDA(cudaMemcpyAsync(out, c->out_stage.p, bytes, cudaMemcpyDeviceToHost, c->stream));
    SOAP_CUDA(cudaStreamSynchronize(c->stream));
    return SOAP_OK;
}

}  // extern "C"

static soap_status active_phases_impl(soap_ctx* c, const soap_region* regions, int32_t n_regions,
                                      const double* phases, int32_t n_phases, const double* radii,
                                      uint32_t effects, int32_t precision, void* out, int out_on_device) {
    if (!c || !out) { set_error("ctx or out is NULL"); return SOAP_EINVAL; }
    ActiveArgs A;
    SOAP_TRY(check_active(c, regions, n_regions, phases, n_phases, effects, precision, A));
    if (radii)
        for (int64_t i = 0; i < (int64_t)n_phases * n_regions; i++)
            if (!(radii[i] >= 0.0 && radii[i] <= 1.0)) {
                set_error("radii[%lld] = %g outside [0, 1]", (long long)i, radii[i]); return SOAP_EINVAL;
            }
    int n_eff = __builtin_popcount(effects);
    size_t esz = precision == SOAP_FP64 ? 8 : 4;
    size_t bytes = (size_t)n_eff * (size_t)n_phases * (size_t)c->n_px * esz;
    if (n_phases == 0) return SOAP_OK;
    void* dst = out;
    if (!out_on_device) {
        SOAP_TRY(ensure(c->out_stage, bytes));
        dst = c->out_stage.p;
    }
    void* raw = dst;                               // before the instrument's line-spread function
    if (c->lsf_K >= 0) {
        SOAP_TRY(ensure(c->lsf_tmp, bytes));
        raw = c->lsf_tmp.p;
    }
    SOAP_TRY(toeplitz_active(c, A.rd.data(), n_regions, A.ctemp, A.ctype, A.n_class, phases, n_phases,
                             effects, precision, raw, radii));
    if (c->lsf_K >= 0) SOAP_TRY(launch_lsf(c, raw, dst, precision != SOAP_FP64, (int64_t)n_eff * n_phases));
    if (!out_on_device) {
        SOAP_CUDA(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
        SOAP_CUDA(cudaStreamSynchronize(c->stream));
        SOAP_TRY(check_flags(c));
    }
    return SOAP_OK;
}

// Area (MSH) of an evolving region at time t (days): the laws and readings of Sect. 4.2.1 as
// stated in soap.h.
static double evolution_area(const soap_region_evolution& e, double t) {
    switch (e.law) {
        case SOAP_EVOLVE_LINEAR_GROWTH: return e.area0_msh + e.rate_msh_per_day * std::max(t, 0.0);
        case SOAP_EVOLVE_LINEAR_DECAY: return std::max(0.0, e.area0_msh - e.rate_msh_per_day * std::max(t, 0.0));
        case SOAP_EVOLVE_ASYM_GAUSSIAN: {
            const double tot = e.fwhm_day / std::sqrt(2.0 * std::log(2.0));
            const double s = t < e.t_peak_day ? tot * (1.0 - e.asymmetry) / 2.0 : tot * (1.0 + e.asymmetry) / 2.0;
            const double u = (t - e.t_peak_day) / s;
            return e.area0_msh * std::exp(-0.5 * u * u);
        }
        default: return -1.0;
    }
}

extern "C" {

soap_status soap_evolve_radii(const soap_region_evolution* evo, const soap_region* regions, int32_t n_regions,
                              const double* times_day, int32_t n_times, double* radii) {
    clear_error();
    if (n_regions < 0 || n_times < 0) { set_error("negative count"); return SOAP_EINVAL; }
    if ((n_regions > 0 && (!evo || !regions)) || (n_times > 0 && !times_day) ||
        (n_regions > 0 && n_times > 0 && !radii)) {
        set_error("NULL argument"); return SOAP_EINVAL;
    }
    for (int q = 0; q < n_regions; q++) {
        const soap_region_evolution& e = evo[q];
        if (e.law < SOAP_EVOLVE_NONE || e.law > SOAP_EVOLVE_ASYM_GAUSSIAN) { set_error("evo[%d].law unknown", q); return SOAP_EINVAL; }
        if (e.law != SOAP_EVOLVE_NONE &&
            (!is_finite(e.area0_msh) || e.area0_msh < 0 || !is_finite(e.rate_msh_per_day) ||
             !is_finite(e.t_peak_day) || (e.law == SOAP_EVOLVE_ASYM_GAUSSIAN &&
                                           (!(e.fwhm_day > 0) || !(std::fabs(e.asymmetry) < 1.0))))) {
            set_error("evo[%d] has an invalid parameter", q); return SOAP_EINVAL;
        }
    }
    for (int p = 0; p < n_times; p++) {
        if (!is_finite(times_day[p])) { set_error("times_day[%d] not finite", p); return SOAP_EINVAL; }
        for (int q = 0; q < n_regions; q++) {
            const soap_region_evolution& e = evo[q];
            double r = regions[q].radius_rstar;
            if (e.law != SOAP_EVOLVE_NONE) r = std::sqrt(evolution_area(e, times_day[p]) * 1e-6);
            radii[(int64_t)p * n_regions + q] = std::min(r, 1.0);
        }
    }
    return SOAP_OK;
}

soap_status soap_active_phases(soap_ctx* c, const soap_region* regions, int32_t n_regions,
                               const double* phases, int32_t n_phases, uint32_t effects,
                               int32_t precision, void* out, int out_on_device) {
    clear_error();
    return active_phases_impl(c, regions, n_regions, phases, n_phases, nullptr, effects, precision, out,
                              out_on_device);
}

soap_status soap_active_phases_radii(soap_ctx* c, const soap_region* regions, int32_t n_regions,
                                     const double* phases, int32_t n_phases, const double* radii,
                                     uint32_t effects, int32_t precision, void* out, int out_on_device) {
    clear_error();
    if (!radii && n_regions > 0 && n_phases > 0) { set_error("radii is NULL"); return SOAP_EINVAL; }
    return active_phases_impl(c, regions, n_regions, phases, n_phases, radii, effects, precision, out,
                              out_on_device);
}

soap_status soap_active_rv(soap_ctx* c, const soap_region* regions, int32_t n_regions,
                           const double* phases, int32_t n_phases, uint32_t effect,
                           int32_t precision, const double* mask_lambda, const double* mask_weight,
                           int32_t n_lines, double mask_width_kms, double v_lo, double v_step,
                           int32_t n_v, void* spectra_out, double* rv_kms, int out_on_device) {
    clear_error();
    if (!c || !rv_kms) { set_error("ctx or rv_kms is NULL"); return SOAP_EINVAL; }
    if (effect != SOAP_EFFECT_FLUX && effect != SOAP_EFFECT_BCONV && effect != SOAP_EFFECT_TOT) {
        set_error("effect must be exactly one of SOAP_EFFECT_*"); return SOAP_EINVAL;
    }
    ActiveArgs A;
    SOAP_TRY(check_active(c, regions, n_regions, phases, n_phases, effect, precision, A));
    SOAP_TRY(check_rv(c, mask_lambda, mask_weight, n_lines, mask_width_kms, v_lo, v_step, n_v));
    if (n_phases == 0) return SOAP_OK;
    const int f32 = precision != SOAP_FP64;
    const bool ccf_tc = precision == SOAP_BF16X3 || (precision == SOAP_FP32 && c->ccf_tc);
    const size_t sbytes = (size_t)n_phases * (size_t)c->n_px * (f32 ? 4 : 8);
    if (out_on_device) {
        void* sp = spectra_out;
        if (!sp) {
            SOAP_TRY(ensure(c->out_stage, sbytes));
            sp = c->out_stage.p;
        }
        SOAP_TRY(active_lsf(c, A, n_regions, phases, n_phases, effect, precision, sp, sbytes));
        return rv_ccf_run(c, sp, f32, n_phases, mask_lambda, mask_weight, n_lines, mask_width_kms,
                          v_lo, v_step, n_v, rv_kms, nullptr, nullptr, ccf_tc);
    }
    // host results: computed into one of two alternating device buffers; the spectra go to the
    // host on out_stream while the CCF runs, the RVs after the fit
    SOAP_TRY(ensure_pipeline(c));
    const int o = c->dn_next;
    c->dn_next ^= 1;
    const size_t o_rv = (sbytes + 255) / 256 * 256;
    soap::DevBuf& d = c->dn_stage[o];
    SOAP_TRY(ensure(d, o_rv + (size_t)n_phases * 8));
    void* spec_d = d.p;
    double* rv_d = reinterpret_cast<double*>(d.as<char>() + o_rv);
    SOAP_CUDA(cudaStreamWaitEvent(c->stream, c->dn_free[o], 0));        // its last copy out is done
    SOAP_TRY(active_lsf(c, A, n_regions, phases, n_phases, effect, precision, spec_d, sbytes));
    if (spectra_out) {
        SOAP_CUDA(cudaEventRecord(c->dn_spec[o], c->stream));
        SOAP_CUDA(cudaStreamWaitEvent(c->out_stream, c->dn_spec[o], 0));
        SOAP_CUDA(cudaMemcpyAsync(spectra_out, spec_d, sbytes, cudaMemcpyDeviceToHost, c->out_stream));
    }
    SOAP_TRY(rv_ccf_run(c, spec_d, f32, n_phases, mask_lambda, mask_weight, n_lines, mask_width_kms,
                        v_lo, v_step, n_v, rv_d, nullptr, nullptr, ccf_tc));
    SOAP_CUDA(cudaEventRecord(c->dn_rv[o], c->stream));
    SOAP_CUDA(cudaStreamWaitEvent(c->out_stream, c->dn_rv[o], 0));
    SOAP_CUDA(cudaMemcpyAsync(rv_kms, rv_d, (size_t)n_phases * 8, cudaMemcpyDeviceToHost, c->out_stream));
    SOAP_CUDA(cudaEventRecord(c->dn_free[o], c->out_stream));
    if (!c->host_async) {
        SOAP_CUDA(cudaStreamSynchronize(c->out_stream));
        SOAP_TRY(check_flags(c));
    }
    return SOAP_OK;
}

soap_status soap_rv_ccf(soap_ctx* c, const void* spectra, int32_t spectra_f32, int32_t n_spec,
                        int spectra_on_device, const double* mask_lambda,
                        const double* mask_weight, int32_t n_lines, double mask_width_kms,
                        double v_lo, double v_step, int32_t n_v, double* rv_kms,
                        double* fit_params, double* ccf_out, int out_on_device) {
    clear_error();
    if (!c || !spectra || !mask_lambda || !mask_weight || !rv_kms) {
        set_error("NULL argument"); return SOAP_EINVAL;
    }
    if (n_spec < 0) { set_error("need n_spec >= 0"); return SOAP_EINVAL; }
    if (spectra_f32 < 0 || spectra_f32 > 2) { set_error("spectra_f32 must be 0, 1 or 2"); return SOAP_EINVAL; }
    SOAP_TRY(check_rv(c, mask_lambda, mask_weight, n_lines, mask_width_kms, v_lo, v_step, n_v));
    if (n_spec == 0) return SOAP_OK;
    size_t esz = spectra_f32 ? 4 : 8;
    size_t sbytes = (size_t)n_spec * (size_t)c->n_px * esz;
    const void* dspec = spectra;
    if (!spectra_on_device) {
        SOAP_TRY(ensure(c->stage_in, sbytes));
        SOAP_CUDA(cudaMemcpyAsync(c->stage_in.p, spectra, sbytes, cudaMemcpyHostToDevice, c->stream));
        dspec = c->stage_in.p;
    }
    double* rv_d = rv_kms;
    double* fit_d = fit_params;
    double* ccf_d = ccf_out;
    size_t o_rv = 0, o_fit = 0, o_ccf = 0, total = 0;
    if (!out_on_device) {
        o_rv = 0;
        o_fit = o_rv + (size_t)n_spec * 8;
        o_ccf = o_fit + (size_t)n_spec * 32;
        total = o_ccf + (size_t)n_spec * n_v * 8;
        SOAP_TRY(ensure(c->out_stage, total));
        char* base = c->out_stage.as<char>();
        rv_d = (double*)(base + o_rv);
        fit_d = (double*)(base + o_fit);
        ccf_d = (double*)(base + o_ccf);
    }
    SOAP_TRY(rv_ccf_run(c, dspec, spectra_f32 ? 1 : 0, n_spec, mask_lambda, mask_weight, n_lines,
                        mask_width_kms, v_lo, v_step, n_v, rv_d, fit_d, ccf_d, spectra_f32 == 2));
    if (!out_on_device) {
        SOAP_CUDA(cudaMemcpyAsync(rv_kms, rv_d, (size_t)n_spec * 8, cudaMemcpyDeviceToHost, c->stream));
        if (fit_params)
            SOAP_CUDA(cudaMemcpyAsync(fit_params, fit_d, (size_t)n_spec * 32, cudaMemcpyDeviceToHost, c->stream));
        if (ccf_out)
            SOAP_CUDA(cudaMemcpyAsync(ccf_out, ccf_d, (size_t)n_spec * n_v * 8, cudaMemcpyDeviceToHost, c->stream));
        SOAP_CUDA(cudaStreamSynchronize(c->stream));
        // a tensor-core wait that gave up left a partial CCF: report it with the results
        SOAP_TRY(check_flags(c));
    }
    return SOAP_OK;
}

soap_status soap_batch_set_rv(soap_ctx* c, const double* mask_lambda, const double* mask_weight,
                              int32_t n_lines, double mask_width_kms, double v_lo, double v_step,
                              int32_t n_v, double fit_margin_kms, int32_t tensor_cores) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return SOAP_EINVAL; }
    if (!is_finite(fit_margin_kms)) { set_error("fit_margin_kms not finite"); return SOAP_EINVAL; }
    if (tensor_cores != 0 && tensor_cores != 1) { set_error("tensor_cores must be 0 or 1"); return SOAP_EINVAL; }
    if (!mask_lambda || !mask_weight) { set_error("NULL mask"); return SOAP_EINVAL; }
    if (n_lines < 1 || n_v < 5 || n_v > 4096) { set_error("need n_lines >= 1, 5 <= n_v <= 4096"); return SOAP_EINVAL; }
    for (int l = 0; l < n_lines; l++)
        if (!is_finite(mask_lambda[l]) || !(mask_lambda[l] > 0) || !is_finite(mask_weight[l])) {
            set_error("mask line %d invalid", l); return SOAP_EINVAL;
        }
    if (!is_finite(mask_width_kms) || !(mask_width_kms > 0) || !is_finite(v_lo) || !is_finite(v_step) || !(v_step > 0)) {
        set_error("mask width / velocity grid invalid"); return SOAP_EINVAL;
    }
    const double v_hi = v_lo + v_step * (n_v - 1);
    if (!(std::fabs(v_lo) < kCKms) || !(std::fabs(v_hi) < kCKms)) { set_error("velocity grid reaches c"); return SOAP_EINVAL; }
    if (mask_width_kms / (kCKms * c->delta) > 14.0) { set_error("mask box spans more than 14 pixels"); return SOAP_ERANGE; }
    c->b_rv_lambda.assign(mask_lambda, mask_lambda + n_lines);
    c->b_rv_weight.assign(mask_weight, mask_weight + n_lines);
    c->b_rv_width = mask_width_kms;
    c->b_rv_v_lo = v_lo;
    c->b_rv_v_step = v_step;
    c->b_rv_n_v = n_v;
    c->b_rv_margin = fit_margin_kms;
    c->b_rv_tc = tensor_cores;
    c->b_rv_set = true;
    return SOAP_OK;
}

soap_status soap_active_batch(soap_ctx* c, const soap_batch_item* items, int32_t n_items,
                              const soap_region* regions, int32_t n_regions, const double* phases,
                              int32_t n_phases, int32_t output, float* out, double* rv_kms,
                              int out_on_device) {
    clear_error();
    if (!c || !out) { set_error("ctx or out is NULL"); return SOAP_EINVAL; }
    if (output != SOAP_BATCH_SPECTRUM && output != SOAP_BATCH_RESIDUAL) { set_error("unknown output %d", output); return SOAP_EINVAL; }
    if (rv_kms && output != SOAP_BATCH_SPECTRUM) {
        set_error("radial velocities need output = SOAP_BATCH_SPECTRUM (residual rows are not spectra)");
        return SOAP_EINVAL;
    }
    if (rv_kms && !c->b_rv_set) { set_error("no mask for the batched RVs (soap_batch_set_rv)"); return SOAP_ESTATE; }
    if (n_items < 0 || n_regions < 0 || n_phases < 0) { set_error("negative count"); return SOAP_EINVAL; }
    if ((n_items > 0 && !items) || (n_regions > 0 && !regions) || (n_phases > 0 && !phases)) {
        set_error("items, regions or phases is NULL"); return SOAP_EINVAL;
    }
    int variant = c->b_variant;
    if (variant < 0) {
        // no chosen variant: blocks no wider than the items' phase counts (1, 2, else 4 phases)
        int max_np = 0;
        for (int k = 0; k < n_items; k++) max_np = std::max(max_np, (int)items[k].n_phases);
        variant = batch_default_variant(max_np);
    }
    const size_t bytes = (size_t)n_phases * (size_t)c->n_px * sizeof(float);
    const size_t rv_off = (bytes + 255) / 256 * 256;
    float* dst = out;
    double* rv_dst = rv_kms;
    if (!out_on_device && bytes > 0) {
        SOAP_TRY(ensure(c->out_stage, rv_off + (rv_kms ? (size_t)n_phases * 8 : 0)));
        dst = c->out_stage.as<float>();
        if (rv_kms) rv_dst = reinterpret_cast<double*>(c->out_stage.as<char>() + rv_off);
    }
    SOAP_TRY(batch_run(c, items, n_items, regions, n_regions, phases, n_phases, variant,
                       output == SOAP_BATCH_RESIDUAL, dst, rv_dst));
    if (!out_on_device && bytes > 0) {
        SOAP_CUDA(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
        if (rv_kms)
            SOAP_CUDA(cudaMemcpyAsync(rv_kms, rv_dst, (size_t)n_phases * 8, cudaMemcpyDeviceToHost, c->stream));
        SOAP_CUDA(cudaStreamSynchronize(c->stream));
        SOAP_TRY(check_flags(c));
    }
    return SOAP_OK;
}

soap_status soap_batch_num_variants(int32_t* n) {
    clear_error();
    if (!n) { set_error("n is NULL"); return SOAP_EINVAL; }
    *n = batch_num_variants();
    return SOAP_OK;
}

soap_status soap_batch_variant_info(int32_t variant, int32_t* phases_per_block, int32_t* px_per_thread) {
    clear_error();
    if (!phases_per_block || !px_per_thread) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (variant < 0 || variant >= batch_num_variants()) { set_error("variant %d outside 0..%d", variant, batch_num_variants() - 1); return SOAP_ERANGE; }
    int pb = 0, r = 0;
    batch_variant_info(variant, &pb, &r);
    *phases_per_block = pb;
    *px_per_thread = r;
    return SOAP_OK;
}

soap_status soap_batch_set_variant(soap_ctx* c, int32_t variant) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return SOAP_EINVAL; }
    if (variant < -1 || variant >= batch_num_variants()) { set_error("variant %d outside -1..%d", variant, batch_num_variants() - 1); return SOAP_ERANGE; }
    c->b_variant = variant;
    return SOAP_OK;
}

soap_status soap_batch_get_variant(const soap_ctx* c, int32_t* variant) {
    clear_error();
    if (!c || !variant) { set_error("NULL argument"); return SOAP_EINVAL; }
    *variant = c->b_variant;
    return SOAP_OK;
}

soap_status soap_batch_autotune(soap_ctx* c, const soap_batch_item* items, int32_t n_items,
                                const soap_region* regions, int32_t n_regions, const double* phases,
                                int32_t n_phases, float* out, int32_t reps, float* ms, int32_t* best_variant) {
    clear_error();
    if (!c || !out || !best_variant) { set_error("NULL argument"); return SOAP_EINVAL; }
    if (reps < 1) { set_error("reps must be >= 1"); return SOAP_EINVAL; }
    const int nv = batch_num_variants();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SOAP_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); set_error("cudaEventCreate failed"); return SOAP_ECUDA; }
    soap_status st = SOAP_OK;
    int best = -1;
    float best_ms = 0;
    for (int v = 0; v < nv && st == SOAP_OK; v++) {
        st = batch_run(c, items, n_items, regions, n_regions, phases, n_phases, v, 0, out);   // capture + warm
        if (st != SOAP_OK) break;
        if (cudaEventRecord(e0, c->stream) != cudaSuccess) { st = SOAP_ECUDA; break; }
        for (int k = 0; k < reps && st == SOAP_OK; k++)
            st = batch_run(c, items, n_items, regions, n_regions, phases, n_phases, v, 0, out);
        if (st != SOAP_OK) break;
        float t = 0;
        if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            set_error("autotune timing failed"); st = SOAP_ECUDA; break;
        }
        t /= (float)reps;
        if (ms) ms[v] = t;
        if (best < 0 || t < best_ms) { best = v; best_ms = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SOAP_OK) return st;
    SOAP_CUDA(cudaStreamSynchronize(c->stream));
    SOAP_TRY(check_flags(c));
    c->b_variant = best;
    *best_variant = best;
    return SOAP_OK;
}

void soap_free(soap_ctx* c) {
    if (!c) return;
    sync_all(c);
    destroy_pipeline(c);
    destroy_events(c);
    batch_release(c);
    free_ctx_memory(c);
    delete c;
}

}  // extern "C"
