// batch.cu -- batched persistent form: many independent active-region configurations of one
// star type (shared local spectra, disk grid, limb darkening, mu table), each with its own
// vsini, inclination, regions and phases, computed by one CUDA-graph launch.
//
// Without differential rotation a cell's velocity is vsini x, so a configuration's pixel
// shifts depend only on the column x of the cell: per configuration, a column table (tap j,
// weight w as a 32-bit fraction) replaces per-cell geometry, and the quiet velocity kernels
// come from per-(column, mu bin) intensity sums split by w in exact integer arithmetic.
//
// Stages (all on the context's stream, captured once per batch shape into a CUDA graph):
//  1 k_batch_star     per column: I per cell in fixed point, per-(column, bin) sums
//  2 k_batch_items    per configuration: column table, quiet kernels, quiet job table
//  3 k_batch_quiet    quiet spectrum per configuration (Toeplitz contraction)
//  4 k_batch_regions  region centres / cell boxes per (phase, region)
//  5 k_batch_hist     InfoMap + per-phase kernels; the last block of each phase block builds
//                     its job table
//  6 k_batch_contract persistent: blocks take phase blocks (all pixel tiles of one) from an
//                     atomic ticket, in an order sorted by estimated cost (largest first)
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "contract_dev.cuh"

namespace soap {

struct BatchItemDev {
    double vsini, incl_deg;
    int first_region, n_regions, first_phase, n_phases;
    int n_cls;                           // the item's region classes (type, temperature)
    int cls_type[SOAP_MAX_CLASSES];
    float cls_a[SOAP_MAX_CLASSES];       // h c / (lambda_s k T_class)
};

struct PBlockDev {
    int item, first_phase, np, pad;
};

// Split an integer intensity into its two taps: k1 = floor(|I| w / 2^32) (sign of I),
// k0 = I - k1 (exact sum).  With |I| = hi 2^32 + lo, floor(|I| w / 2^32) = hi w + umulhi(lo, w):
// 32-bit multiplies only.
__device__ __forceinline__ void split_fx(long long I, unsigned int wfx, long long& k0, long long& k1) {
    const unsigned long long a = I >= 0 ? (unsigned long long)I : (unsigned long long)(-I);
    const unsigned int hi = (unsigned int)(a >> 32), lo = (unsigned int)a;
    const unsigned long long h = (unsigned long long)hi * wfx + __umulhi(lo, wfx);
    k1 = I >= 0 ? (long long)h : -(long long)h;
    k0 = I - k1;
}

// Stage 1: block per column i.  I_fx per cell and IB[i][b] = sum_j I_fx(i, j) [bin = b].
__global__ void k_batch_star(int N, int n_mu, const double* __restrict__ cell_I,
                             const int32_t* __restrict__ cell_bin, double scale,
                             long long* __restrict__ cell_Ifx, long long* __restrict__ IB) {
    extern __shared__ long long sb[];
    const int i = blockIdx.x;
    for (int t = threadIdx.x; t < n_mu; t += blockDim.x) sb[t] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const int64_t c = (int64_t)j * N + i;
        const int b = cell_bin[c];
        long long v = 0;
        if (b >= 0) {
            v = __double2ll_rn(cell_I[c] * scale);
            atomicAdd((unsigned long long*)&sb[b], (unsigned long long)v);
        }
        cell_Ifx[c] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n_mu; t += blockDim.x) IB[(int64_t)i * n_mu + t] = sb[t];
}

// Stage 2: block per configuration.
__global__ void k_batch_items(int N, int n_mu, int n_taps, int tap_min, double inv_c, double inv_delta,
                              double delta, double inv_expm1_delta, const BatchItemDev* __restrict__ items,
                              const long long* __restrict__ IB, int* __restrict__ colj,
                              unsigned int* __restrict__ colw, long long* __restrict__ kq,
                              long long* qtoff, int* qgs, float* qc32, int q_max_taps, double inv_scale,
                              int fx_bits, int64_t row_len, int64_t pad, unsigned int* flags) {
    extern __shared__ long long hist[];                  // [n_mu][n_taps]
    const int it = blockIdx.x;
    const int nb = n_mu * n_taps;
    const double vsini = items[it].vsini;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double x = (double)(2 * i + 1 - N) / (double)N;
        const double beta = vsini * x * inv_c;
        const double ab = fabs(beta) <= 1e-3 ? atanh_small(beta) : atanh(beta);
        const double jd = ceil(ab * inv_delta);
        int jt = (int)jd;
        const double e = fma(jd, delta, -ab);
        double w = (delta <= 1e-3 ? expm1_small(e) : expm1(e)) * inv_expm1_delta;
        w = fmin(fmax(w, 0.0), 1.0);
        const unsigned int wfx = (unsigned int)fmin(rint(w * 4294967296.0), 4294967295.0);
        if (jt - 1 < tap_min || jt > tap_min + n_taps - 1) {
            atomicOr(flags, kFlagTapRange);
            jt = jt < tap_min + 1 ? tap_min + 1 : tap_min + n_taps - 1;
        }
        colj[(int64_t)it * N + i] = jt;
        colw[(int64_t)it * N + i] = wfx;
        const int kk = jt - tap_min;
        for (int b = 0; b < n_mu; b++) {
            const long long ib = IB[(int64_t)i * n_mu + b];
            if (ib == 0) continue;
            long long k0, k1;
            split_fx(ib, wfx, k0, k1);
            atomicAdd((unsigned long long*)&hist[b * n_taps + kk], (unsigned long long)k0);
            atomicAdd((unsigned long long*)&hist[b * n_taps + kk - 1], (unsigned long long)k1);
        }
    }
    __syncthreads();
    long long* dst = kq + (int64_t)it * nb;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) dst[t] = hist[t];
    __threadfence_block();
    __syncthreads();
    build_taps_dev(dst, 0, 1, 1, n_mu, n_taps, tap_min, 1, 0, inv_scale, fx_bits, row_len, pad,
                   qtoff + (int64_t)it * q_max_taps, qgs + (int64_t)it * 2, nullptr,
                   qc32 + (int64_t)it * q_max_taps, q_max_taps, hist, flags);
}

// Stage 3: grid (tiles, configurations).
template <int R, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_batch_quiet(int64_t n_px, Rows<float> rows, const long long* __restrict__ qtoff, const int* __restrict__ qgs,
              const float* __restrict__ qc32, int q_max_taps, float* __restrict__ fq) {
    const int it = blockIdx.y;
    const TableContrast<float> con{nullptr, n_px, ClassTypes{}};
    contract_tile<float, 1, R, THREADS>(n_px, rows, qtoff + (int64_t)it * q_max_taps, qgs + (int64_t)it * 2, 1,
                                        qc32 + (int64_t)it * q_max_taps, con, nullptr, SOAP_EFFECT_TOT,
                                        blockIdx.x, 1, fq + (int64_t)it * n_px);
}

// Stage 4: thread per (phase, region slot).
__global__ void k_batch_regions(int N, int n_phases, int max_r, const int* __restrict__ phase_item,
                                const BatchItemDev* __restrict__ items, const RegionDev* __restrict__ regs,
                                const double* __restrict__ phases, RegionGeo* __restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_phases * max_r) return;
    const int p = (int)(t / max_r), q = (int)(t % max_r);
    const BatchItemDev it = items[phase_item[p]];
    if (q >= it.n_regions) return;
    out[t] = region_geometry(N, regs[it.first_region + q], phases[p], it.incl_deg, 0.0);
}

// Stage 5: block per phase.  Owned cells add their integer intensity split by their column's
// weight into the block's kernels (shared memory when they fit, stored whole afterwards; else
// global atomics into zeroed memory); the last block of a phase block builds its job table.
__global__ void k_batch_hist(int N, int max_r, const int* __restrict__ phase_item,
                             const int* __restrict__ phase_block, const BatchItemDev* __restrict__ items,
                             const PBlockDev* __restrict__ pblocks, const RegionGeo* __restrict__ geo,
                             const double* __restrict__ cell_mu, const float* __restrict__ cell_mu32,
                             const int32_t* __restrict__ cell_bin, const long long* __restrict__ cell_Ifx,
                             const int* __restrict__ colj, const unsigned int* __restrict__ colw,
                             int tap_min, int n_taps, int n_mu, int n_class, long long* kfix, int use_smem,
                             int PB, double inv_scale, int fx_bits, int64_t row_len, int64_t pad, long long* toff,
                             int* gstart,
                             float* c32, int max_taps, int* counters, int taps_smem, unsigned int* flags,
                             const double* __restrict__ cell_x) {
    __shared__ RegionGeo sg[SOAP_MAX_REGIONS];
    extern __shared__ long long hist_sm[];
    const int p = blockIdx.x;
    const int it = phase_item[p];
    const int nr = items[it].n_regions;
    const int nb = n_class * n_mu * n_taps;
    long long* gdst = kfix + (int64_t)p * nb;
    long long* hist = use_smem ? hist_sm : gdst;
    if (threadIdx.x < nr) sg[threadIdx.x] = geo[(int64_t)p * max_r + threadIdx.x];
    if (use_smem)
        for (int t = threadIdx.x; t < nb; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    const int* cj = colj + (int64_t)it * N;
    const unsigned int* cw = colw + (int64_t)it * N;
    const float invN = 1.0f / small_int_to_float(N);
    for (int r = 0; r < nr; r++) {
        const int i0 = sg[r].box[0], i1 = sg[r].box[1], j0 = sg[r].box[2], j1 = sg[r].box[3];
        if (i1 < i0 || j1 < j0) continue;
        const int wdt = i1 - i0 + 1;
        const int area = wdt * (j1 - j0 + 1);                  // <= N^2 < 2^31
        BoxWalk wk((int)threadIdx.x, (int)blockDim.x, wdt);
        for (int t = threadIdx.x; t < area; t += blockDim.x, wk.next()) {
            const int i = i0 + wk.col, jj = j0 + wk.row;
            if (in_earlier_box(sg, r, i, jj)) continue;
            const int c = jj * N + i;                          // N^2 < 2^31
            const int b = cell_bin[c];
            if (b < 0) continue;
            const int owner = cell_owner(sg, nr, N, invN, i, jj, cell_mu32[c], cell_mu, c, cell_x);
            if (owner < 0) continue;
            const int kk = cj[i] - tap_min;
            if (kk < 1 || kk >= n_taps) { atomicOr(flags, kFlagTapRange); continue; }
            long long k0, k1;
            split_fx(cell_Ifx[c], cw[i], k0, k1);
            long long* h = hist + (sg[owner].cls * n_mu + b) * n_taps;
            atomicAdd((unsigned long long*)&h[kk], (unsigned long long)k0);
            atomicAdd((unsigned long long*)&h[kk - 1], (unsigned long long)k1);
        }
    }
    if (use_smem) {
        __syncthreads();
        for (int t = threadIdx.x; t < nb; t += blockDim.x) gdst[t] = hist[t];
    }
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    const int pbk = phase_block[p];
    const PBlockDev pbd = pblocks[pbk];
    if (threadIdx.x == 0) {
        const int t = atomicAdd(&counters[pbk], 1);
        s_last = t == pbd.np - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        // tables of the classes only (mode 2): the contraction folds the quiet rows into their operands
        build_taps_dev(kfix + (int64_t)pbd.first_phase * nb, 0, pbd.np, n_class, n_mu, n_taps, tap_min, PB, 2,
                       inv_scale, fx_bits, row_len, pad, toff + (int64_t)pbk * max_taps, gstart + (int64_t)pbk * (n_class + 1),
                       nullptr, c32 + (int64_t)pbk * max_taps * PB, max_taps, taps_smem ? hist_sm : nullptr, flags);
    }
}

// Stage 6: persistent.  A unit is one phase block over all pixel tiles; blocks take the next
// unit in `order` with an atomic ticket until none is left (no block waits on another).  The
// contrast of the item's classes is evaluated per pixel (Planck ratio), so items may carry any
// temperatures.  fq == nullptr: residual output F - F_q.
template <int PB, int R, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_batch_contract(int64_t n_px, Rows<float> rows, const long long* __restrict__ toff, const int* __restrict__ gstart,
                 int G, int max_taps, const float* __restrict__ c32, const BatchItemDev* __restrict__ items,
                 float aq, float fd, const float* __restrict__ fq, const PBlockDev* __restrict__ pblocks,
                 const int* __restrict__ order, int n_units, int n_tiles, unsigned int* ticket,
                 float* __restrict__ out) {
    __shared__ int s_u;
    while (true) {
        if (threadIdx.x == 0) s_u = (int)atomicAdd(ticket, 1u);
        __syncthreads();
        const int u = s_u;
        __syncthreads();
        if (u >= n_units) break;
        const int pbk = order[u];
        const PBlockDev pb = pblocks[pbk];
        const long long* tt = toff + (int64_t)pbk * max_taps;
        const int* gs = gstart + (int64_t)pbk * (G + 1);
        const float* cb = c32 + (int64_t)pbk * max_taps * PB;
        const float* fqi = fq ? fq + (int64_t)pb.item * n_px : nullptr;
        float* orow = out + (int64_t)pb.first_phase * n_px;
        const PlanckContrast32 con{aq, fd, items[pb.item].cls_type, items[pb.item].cls_a};
        for (int tile = 0; tile < n_tiles; tile++)
            contract_tile_fold32<PB, R, THREADS, SOAP_EFFECT_TOT>(n_px, rows, tt, gs, G, cb, con, fqi, tile, pb.np,
                                                                  orow);
    }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
constexpr int kBatchThreads = 128;

// Variants the autotuner chooses from: (phases per block, pixels per thread).
struct BatchVariant {
    int PB, R;
};
static const BatchVariant kVariants[] = {{1, 4}, {2, 4}, {4, 2}, {4, 4}, {8, 2}, {8, 4}, {16, 2}, {16, 4}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
constexpr int kDefaultVariant = 3;

// Sizes of one batch, fixed by the host preparation and baked into the captured graph.
struct BatchShape {
    int n_items, n_phases, max_r, n_pblocks, n_units, n_tiles, variant, n_class, residual;
    int G, max_taps;
    int64_t nbk;               // per-phase kernel size n_class * n_mu * n_taps
    int use_smem, taps_smem;
    size_t hist_smem;
};

// h c / (lambda_s k T): the Planck exponent at the first grid wavelength.
static double planck_aq(const soap_ctx* c, double temp) {
    return kPlanckH * kLightSI / kBoltzmann * 1e10 / (c->lam_s * temp);
}
static double planck_aq(const soap_ctx* c) { return planck_aq(c, c->t_quiet); }

template <int PB, int R>
static soap_status launch_batch_contract(soap_ctx* c, const BatchShape& b, const float* a0, const float* a1,
                                         float* out) {
    Rows<float> rows;
    rows.q = c->q32; rows.a[0] = a0; rows.a[1] = a1;
    int dev = 0, sms = 152, per_sm = 4;
    SOAP_CUDA(cudaGetDevice(&dev));
    SOAP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SOAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_contract<PB, R, kBatchThreads>,
                                                            kBatchThreads, 0));
    const int grid = std::max(1, std::min(b.n_units, sms * std::max(1, per_sm)));
    SOAP_TIMED(c, SOAP_TIMER_CONTRACT,
               k_batch_contract<PB, R, kBatchThreads><<<grid, kBatchThreads, 0, c->stream>>>(
                   c->n_px, rows, c->b_toff.as<long long>(), c->b_gstart.as<int>(), b.G, b.max_taps,
                   c->b_coefs.as<float>(), c->b_items.as<BatchItemDev>(), (float)planck_aq(c), (float)c->delta,
                   b.residual ? nullptr : c->b_fq.as<float>(), c->b_pblocks.as<PBlockDev>(), c->b_order.as<int>(),
                   b.n_units, b.n_tiles, c->b_ticket.as<unsigned int>(), out);
               SOAP_LAUNCHED(c));
    return SOAP_OK;
}

// Enqueue stages 1-6 (and, with rv, 7: CCF, reduction and fits of the output rows) on the
// context's stream for a batch whose inputs are already on the device.
static soap_status enqueue_batch(soap_ctx* c, const BatchShape& b, float* out, double* rv, const CcfPlan* rvp) {
    const int N = c->N;
    const int q_max_taps = c->n_mu * c->n_taps;
    const double scale = std::ldexp(1.0, c->fx_bits);
    const double inv_scale = std::ldexp(1.0, -c->fx_bits);
    // 1 star
    SOAP_TIMED(c, SOAP_TIMER_GEOMETRY,
               k_batch_star<<<N, 128, c->n_mu * sizeof(long long), c->stream>>>(
                   N, c->n_mu, c->cell_I, c->cell_bin, scale, c->b_cellIfx.as<long long>(), c->b_IB.as<long long>());
               SOAP_LAUNCHED(c));
    // 2 configurations: column tables, quiet kernels and job tables
    const size_t smem_q = (size_t)c->n_mu * c->n_taps * sizeof(long long);
    SOAP_CUDA(cudaFuncSetAttribute(k_batch_items, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_q));
    SOAP_TIMED(c, SOAP_TIMER_GEOMETRY,
               k_batch_items<<<b.n_items, 128, smem_q, c->stream>>>(
                   N, c->n_mu, c->n_taps, c->tap_min, 1.0 / kCKms, 1.0 / c->delta, c->delta,
                   1.0 / std::expm1(c->delta), c->b_items.as<BatchItemDev>(), c->b_IB.as<long long>(),
                   c->b_colj.as<int>(), c->b_colw.as<unsigned int>(), c->b_kq.as<long long>(),
                   c->b_qtoff.as<long long>(), c->b_qgs.as<int>(), c->b_qc32.as<float>(), q_max_taps, inv_scale,
                   c->fx_bits, c->row_len, c->pad, c->flags);
               SOAP_LAUNCHED(c));
    // 3 quiet spectra (not needed for residual output)
    if (!b.residual) {
        Rows<float> rows;
        rows.q = c->q32; rows.a[0] = nullptr; rows.a[1] = nullptr;
        const int64_t TILE = 128 * 4;
        dim3 grid((unsigned)((c->n_px + TILE - 1) / TILE), (unsigned)b.n_items);
        SOAP_TIMED(c, SOAP_TIMER_CONTRACT_QUIET,
                   k_batch_quiet<4, 128><<<grid, 128, 0, c->stream>>>(
                       c->n_px, rows, c->b_qtoff.as<long long>(), c->b_qgs.as<int>(), c->b_qc32.as<float>(),
                       q_max_taps, c->b_fq.as<float>());
                   SOAP_LAUNCHED(c));
    }
    // 4 regions
    if (b.max_r > 0) {
        const int64_t nt = (int64_t)b.n_phases * b.max_r;
        SOAP_TIMED(c, SOAP_TIMER_REGIONS,
                   k_batch_regions<<<(unsigned)((nt + 127) / 128), 128, 0, c->stream>>>(
                       N, b.n_phases, b.max_r, c->b_phase_item.as<int>(), c->b_items.as<BatchItemDev>(),
                       c->b_regions.as<RegionDev>(), c->b_phases.as<double>(), c->b_geo.as<RegionGeo>());
                   SOAP_LAUNCHED(c));
    }
    // 5 per-phase kernels + job tables
    if (!b.use_smem)
        SOAP_CUDA(cudaMemsetAsync(c->b_kfix.p, 0, (size_t)b.n_phases * b.nbk * sizeof(long long), c->stream));
    SOAP_CUDA(cudaMemsetAsync(c->b_counters.p, 0, (size_t)b.n_pblocks * sizeof(int), c->stream));
    SOAP_CUDA(cudaFuncSetAttribute(k_batch_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.hist_smem));
    SOAP_TIMED(c, SOAP_TIMER_PHASE_HIST,
               k_batch_hist<<<(unsigned)b.n_phases, 128, b.hist_smem, c->stream>>>(
                   N, std::max(b.max_r, 1), c->b_phase_item.as<int>(), c->b_phase_block.as<int>(),
                   c->b_items.as<BatchItemDev>(), c->b_pblocks.as<PBlockDev>(), c->b_geo.as<RegionGeo>(),
                   c->cell_mu, c->cell_mu32, c->cell_bin, c->b_cellIfx.as<long long>(), c->b_colj.as<int>(),
                   c->b_colw.as<unsigned int>(), c->tap_min, c->n_taps, c->n_mu, b.n_class,
                   c->b_kfix.as<long long>(), b.use_smem, kVariants[b.variant].PB, inv_scale, c->fx_bits, c->row_len,
                   c->pad,
                   c->b_toff.as<long long>(), c->b_gstart.as<int>(), c->b_coefs.as<float>(), b.max_taps,
                   c->b_counters.as<int>(), b.taps_smem, c->flags, c->cell_x);
               SOAP_LAUNCHED(c));
    // 6 persistent contraction
    SOAP_CUDA(cudaMemsetAsync(c->b_ticket.p, 0, sizeof(unsigned int), c->stream));
    const float* a0 = c->active_set[0] ? c->a32[0] : c->a32[1];
    const float* a1 = c->active_set[1] ? c->a32[1] : c->a32[0];
    switch (b.variant) {
        case 0: SOAP_TRY((launch_batch_contract<1, 4>(c, b, a0, a1, out))); break;
        case 1: SOAP_TRY((launch_batch_contract<2, 4>(c, b, a0, a1, out))); break;
        case 2: SOAP_TRY((launch_batch_contract<4, 2>(c, b, a0, a1, out))); break;
        case 3: SOAP_TRY((launch_batch_contract<4, 4>(c, b, a0, a1, out))); break;
        case 4: SOAP_TRY((launch_batch_contract<8, 2>(c, b, a0, a1, out))); break;
        case 5: SOAP_TRY((launch_batch_contract<8, 4>(c, b, a0, a1, out))); break;
        case 6: SOAP_TRY((launch_batch_contract<16, 2>(c, b, a0, a1, out))); break;
        default: SOAP_TRY((launch_batch_contract<16, 4>(c, b, a0, a1, out))); break;
    }
    // 7 radial velocities of the output rows (Sect. 4.1), each fitted in its item's window
    if (rv) SOAP_TRY(ccf_enqueue(c, c->b_ccf, *rvp, out, rv, nullptr, nullptr, c->b_win.as<int>()));
    return SOAP_OK;
}

int batch_num_variants() { return kNumVariants; }

void batch_variant_info(int v, int* pb, int* r) {
    *pb = kVariants[v].PB;
    *r = kVariants[v].R;
}

int batch_default_variant(int max_phases_per_item) {
    if (max_phases_per_item <= 1) return 0;      // (1, 4)
    if (max_phases_per_item == 2) return 1;      // (2, 4)
    return kDefaultVariant;
}

void batch_release(soap_ctx* c) {
    if (c->b_graph_exec) cudaGraphExecDestroy(c->b_graph_exec);
    c->b_graph_exec = nullptr;
    c->b_graph_key.clear();
    DevBuf* bufs[] = {&c->b_items, &c->b_regions, &c->b_phases, &c->b_phase_item, &c->b_phase_block,
                      &c->b_pblocks, &c->b_order, &c->b_cellIfx, &c->b_IB, &c->b_colj, &c->b_colw, &c->b_kq,
                      &c->b_qtoff, &c->b_qgs, &c->b_qc32, &c->b_fq, &c->b_geo, &c->b_kfix,
                      &c->b_counters, &c->b_toff, &c->b_gstart, &c->b_coefs, &c->b_ticket,
                      &c->b_win, &c->b_ccf.tab, &c->b_ccf.tmp, &c->b_ccf.m};
    for (DevBuf* b : bufs) release(*b);
    c->b_ccf.lines_ok = c->b_ccf.m_ok = false;
    c->b_ccf.mask_key.clear();
}

// Host preparation (validation, classes, phase blocks, cost-ordered units, uploads), then the
// graph: captured on the first call with a given shape, replayed on later ones.
soap_status batch_run(soap_ctx* c, const soap_batch_item* items, int n_items, const soap_region* regions,
                      int n_regions, const double* phases, int n_phases, int variant, int residual, float* out,
                      double* rv) {
    SOAP_TRY(join_geometry(c));                        // the cell tables (before any capture)
    if (c->alpha != 0.0) {
        set_error("the batched form needs a star without differential rotation (diff_rot_alpha = 0)");
        return SOAP_EINVAL;
    }
    if (variant < 0 || variant >= kNumVariants) { set_error("unknown batch variant %d", variant); return SOAP_EINVAL; }
    const BatchVariant V = kVariants[variant];
    for (int r = 0; r < n_regions; r++) {
        const soap_region& g = regions[r];
        if (g.type != SOAP_SPOT && g.type != SOAP_FACULA) { set_error("regions[%d].type invalid", r); return SOAP_EINVAL; }
        if (g.reserved != 0) { set_error("regions[%d].reserved must be 0", r); return SOAP_EINVAL; }
        if (!std::isfinite(g.lat_deg) || !std::isfinite(g.lon_deg) || !std::isfinite(g.radius_rstar) ||
            !std::isfinite(g.temp_K)) {
            set_error("regions[%d] has a non-finite field", r); return SOAP_EINVAL;
        }
        if (g.radius_rstar < 0 || g.radius_rstar > 1) { set_error("regions[%d].radius_rstar outside [0,1]", r); return SOAP_EINVAL; }
        if (!(g.temp_K > 0)) { set_error("regions[%d].temp_K must be > 0", r); return SOAP_EINVAL; }
    }
    // each item's regions are copied with the index of their class (type, temperature) among
    // the item's classes, in first-appearance order
    std::vector<RegionDev> rd;
    int n_class = 0;
    bool uses[3] = {false, false, false};
    // configurations, phase ownership, phase blocks and their estimated cost
    std::vector<BatchItemDev> it(std::max(1, n_items));
    std::vector<int> phase_item(std::max(1, n_phases), -1), phase_block(std::max(1, n_phases), -1);
    std::vector<PBlockDev> pbl;
    std::vector<double> pcost;
    int max_r = 0;
    const double vmax = std::fabs(c->vsini);
    for (int k = 0; k < n_items; k++) {
        const soap_batch_item& s = items[k];
        if (!std::isfinite(s.vsini_kms) || std::fabs(s.vsini_kms) > vmax || !std::isfinite(s.incl_deg) ||
            s.incl_deg < 0 || s.incl_deg > 180) {
            set_error("items[%d]: need |vsini| <= the star's vsini (%g km/s) and 0 <= incl <= 180", k, vmax);
            return SOAP_EINVAL;
        }
        if (s.n_regions < 0 || s.n_regions > SOAP_MAX_REGIONS || s.first_region < 0 ||
            (int64_t)s.first_region + s.n_regions > n_regions || s.n_phases < 0 || s.first_phase < 0 ||
            (int64_t)s.first_phase + s.n_phases > n_phases) {
            set_error("items[%d]: region or phase range out of bounds", k); return SOAP_EINVAL;
        }
        double area = 0;
        BatchItemDev d{};
        d.vsini = s.vsini_kms; d.incl_deg = s.incl_deg;
        d.first_region = (int)rd.size(); d.n_regions = s.n_regions;
        d.first_phase = s.first_phase; d.n_phases = s.n_phases;
        double ctemp[SOAP_MAX_CLASSES];
        for (int r = 0; r < s.n_regions; r++) {
            const soap_region& g = regions[s.first_region + r];
            area += g.radius_rstar * g.radius_rstar;
            int cl = -1;
            for (int q = 0; q < d.n_cls; q++)
                if (d.cls_type[q] == g.type && ctemp[q] == g.temp_K) cl = q;
            if (cl < 0) {
                if (d.n_cls == SOAP_MAX_CLASSES) {
                    set_error("items[%d]: more than %d distinct (type, temperature) pairs", k, SOAP_MAX_CLASSES);
                    return SOAP_ERANGE;
                }
                cl = d.n_cls++;
                d.cls_type[cl] = g.type;
                ctemp[cl] = g.temp_K;
                d.cls_a[cl] = (float)planck_aq(c, g.temp_K);
                uses[g.type] = true;
            }
            rd.push_back(RegionDev{g.lat_deg, g.lon_deg, g.radius_rstar, g.temp_K, g.type, cl});
        }
        n_class = std::max(n_class, d.n_cls);
        for (int p = 0; p < s.n_phases; p++) {
            const int q = s.first_phase + p;
            if (phase_item[q] != -1) { set_error("phase %d belongs to two items", q); return SOAP_EINVAL; }
            if (!std::isfinite(phases[q])) { set_error("phases[%d] not finite", q); return SOAP_EINVAL; }
            phase_item[q] = k;
        }
        for (int p0 = 0; p0 < s.n_phases; p0 += V.PB) {
            const int np = std::min(V.PB, s.n_phases - p0);
            for (int p = 0; p < np; p++) phase_block[s.first_phase + p0 + p] = (int)pbl.size();
            pbl.push_back(PBlockDev{k, s.first_phase + p0, np, 0});
            // work of one unit ~ phases x (quiet-row taps + active taps); the active part grows
            // with the spotted area and the velocity spread across it
            pcost.push_back(np * (1.0 + 40.0 * area * (1.0 + std::fabs(s.vsini_kms))));
        }
        max_r = std::max(max_r, s.n_regions);
        it[k] = d;
    }
    if (uses[SOAP_SPOT] && !c->active_set[0]) { set_error("no active spectrum set for spots"); return SOAP_ESTATE; }
    if (uses[SOAP_FACULA] && !c->active_set[0] && !c->active_set[1]) {
        set_error("no active spectrum set for faculae"); return SOAP_ESTATE;
    }
    for (int p = 0; p < n_phases; p++)
        if (phase_item[p] < 0) { set_error("phase %d belongs to no item", p); return SOAP_EINVAL; }
    // fit windows of the RVs: per item the grid velocities with |v| <= |vsini| + margin
    std::vector<int> win;
    if (rv) {
        if (!c->b_rv_set) { set_error("no mask for the batched RVs (soap_batch_set_rv)"); return SOAP_ESTATE; }
        const int nv = c->b_rv_n_v;
        win.resize(2 * (size_t)std::max(1, n_phases));
        for (int k = 0; k < n_items; k++) {
            int k0 = 0, n = nv;
            if (c->b_rv_margin > 0) {
                const double H = std::fabs(items[k].vsini_kms) + c->b_rv_margin;
                const double a = std::ceil((-H - c->b_rv_v_lo) / c->b_rv_v_step - 1e-9);
                const double z = std::floor((H - c->b_rv_v_lo) / c->b_rv_v_step + 1e-9);
                const int lo = (int)std::max(0.0, a), hi = (int)std::min((double)(nv - 1), z);
                k0 = lo;
                n = hi - lo + 1;
            }
            if (n < 5) {
                set_error("items[%d]: its fit window (|v| <= |vsini| + %g km/s) holds %d < 5 grid velocities", k,
                          c->b_rv_margin, std::max(n, 0));
                return SOAP_EINVAL;
            }
            for (int p = 0; p < items[k].n_phases; p++) {
                win[2 * (size_t)(items[k].first_phase + p)] = k0;
                win[2 * (size_t)(items[k].first_phase + p) + 1] = n;
            }
        }
    }
    if (n_items == 0 || n_phases == 0) return SOAP_OK;
    BatchShape b{};
    b.n_items = n_items;
    b.n_phases = n_phases;
    b.max_r = max_r;
    b.n_pblocks = (int)pbl.size();
    b.n_tiles = (int)((c->n_px + kBatchThreads * V.R - 1) / (kBatchThreads * V.R));
    b.n_units = b.n_pblocks;
    b.variant = variant;
    b.n_class = n_class;
    b.residual = residual ? 1 : 0;
    b.G = n_class;                                     // class groups (quiet rows folded in)
    b.max_taps = std::max(b.G, 1) * c->n_mu * c->n_taps;
    b.nbk = (int64_t)n_class * c->n_mu * c->n_taps;
    const size_t hist_bytes = (size_t)b.nbk * sizeof(long long);
    const size_t kslice_bytes = (size_t)V.PB * b.nbk * sizeof(long long);
    b.use_smem = hist_bytes <= 96 * 1024;
    b.taps_smem = kslice_bytes <= 160 * 1024;
    b.hist_smem = std::max(b.use_smem ? hist_bytes : (size_t)0, b.taps_smem ? kslice_bytes : (size_t)0);
    // units: phase blocks, largest estimated cost first
    std::vector<int> border(b.n_pblocks);
    std::iota(border.begin(), border.end(), 0);
    std::stable_sort(border.begin(), border.end(), [&](int x, int y) { return pcost[x] > pcost[y]; });
    const std::vector<int>& order = border;
    // device buffers (grow-only)
    const int N = c->N;
    const size_t n_rd = std::max<size_t>(1, rd.size());
    SOAP_TRY(ensure(c->b_items, (size_t)n_items * sizeof(BatchItemDev)));
    SOAP_TRY(ensure(c->b_regions, n_rd * sizeof(RegionDev)));
    SOAP_TRY(ensure(c->b_phases, (size_t)n_phases * sizeof(double)));
    SOAP_TRY(ensure(c->b_phase_item, (size_t)n_phases * sizeof(int)));
    SOAP_TRY(ensure(c->b_phase_block, (size_t)n_phases * sizeof(int)));
    SOAP_TRY(ensure(c->b_pblocks, (size_t)b.n_pblocks * sizeof(PBlockDev)));
    SOAP_TRY(ensure(c->b_order, (size_t)b.n_units * sizeof(int)));
    SOAP_TRY(ensure(c->b_cellIfx, (size_t)N * N * sizeof(long long)));
    SOAP_TRY(ensure(c->b_IB, (size_t)N * c->n_mu * sizeof(long long)));
    SOAP_TRY(ensure(c->b_colj, (size_t)n_items * N * sizeof(int)));
    SOAP_TRY(ensure(c->b_colw, (size_t)n_items * N * sizeof(unsigned int)));
    SOAP_TRY(ensure(c->b_kq, (size_t)n_items * c->n_mu * c->n_taps * sizeof(long long)));
    SOAP_TRY(ensure(c->b_qtoff, (size_t)n_items * c->n_mu * c->n_taps * sizeof(long long)));
    SOAP_TRY(ensure(c->b_qgs, (size_t)n_items * 2 * sizeof(int)));
    SOAP_TRY(ensure(c->b_qc32, (size_t)n_items * c->n_mu * c->n_taps * sizeof(float)));
    if (!residual) SOAP_TRY(ensure(c->b_fq, (size_t)n_items * c->n_px * sizeof(float)));
    SOAP_TRY(ensure(c->b_geo, (size_t)n_phases * std::max(1, max_r) * sizeof(RegionGeo)));
    SOAP_TRY(ensure(c->b_kfix, (size_t)n_phases * std::max<int64_t>(1, b.nbk) * sizeof(long long)));
    SOAP_TRY(ensure(c->b_counters, (size_t)b.n_pblocks * sizeof(int)));
    SOAP_TRY(ensure(c->b_toff, (size_t)b.n_pblocks * b.max_taps * sizeof(long long)));
    SOAP_TRY(ensure(c->b_gstart, (size_t)b.n_pblocks * (b.G + 1) * sizeof(int)));
    SOAP_TRY(ensure(c->b_coefs, (size_t)b.n_pblocks * b.max_taps * V.PB * sizeof(float)));
    SOAP_TRY(ensure(c->b_ticket, sizeof(unsigned int)));
    // RVs: fit windows, CCF tables and scratch (tables built here, before any capture)
    CcfPlan rvp;
    if (rv) {
        SOAP_TRY(ensure(c->b_win, win.size() * sizeof(int)));
        SOAP_TRY(ccf_prepare(c, c->b_ccf, c->b_rv_lambda.data(), c->b_rv_weight.data(), (int)c->b_rv_lambda.size(),
                             c->b_rv_width, c->b_rv_v_lo, c->b_rv_v_step, c->b_rv_n_v, n_phases, 1, c->b_rv_tc, rvp));
    }
    // inputs (pageable copies: the call returns after the driver has staged them)
    SOAP_CUDA(cudaMemcpyAsync(c->b_items.p, it.data(), (size_t)n_items * sizeof(BatchItemDev), cudaMemcpyHostToDevice, c->stream));
    if (!rd.empty())
        SOAP_CUDA(cudaMemcpyAsync(c->b_regions.p, rd.data(), rd.size() * sizeof(RegionDev), cudaMemcpyHostToDevice, c->stream));
    SOAP_CUDA(cudaMemcpyAsync(c->b_phases.p, phases, (size_t)n_phases * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    SOAP_CUDA(cudaMemcpyAsync(c->b_phase_item.p, phase_item.data(), (size_t)n_phases * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    SOAP_CUDA(cudaMemcpyAsync(c->b_phase_block.p, phase_block.data(), (size_t)n_phases * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    SOAP_CUDA(cudaMemcpyAsync(c->b_pblocks.p, pbl.data(), (size_t)b.n_pblocks * sizeof(PBlockDev), cudaMemcpyHostToDevice, c->stream));
    SOAP_CUDA(cudaMemcpyAsync(c->b_order.p, order.data(), (size_t)b.n_units * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    if (rv)
        SOAP_CUDA(cudaMemcpyAsync(c->b_win.p, win.data(), (size_t)n_phases * 2 * sizeof(int), cudaMemcpyHostToDevice,
                                  c->stream));
    if (c->profiling)      // per-kernel timers need events between the launches: no graph
        return enqueue_batch(c, b, out, rv, &rvp);
    // everything the graph bakes in: sizes, star parameters and pointers
    std::vector<uint64_t> key;
    auto put = [&](uint64_t v) { key.push_back(v); };
    auto putd = [&](double v) { uint64_t u; memcpy(&u, &v, 8); key.push_back(u); };
    auto putp = [&](const void* p) { key.push_back((uint64_t)(uintptr_t)p); };
    put(b.n_items); put(b.n_phases); put(b.max_r); put(b.n_pblocks); put(b.n_units); put(b.n_tiles);
    put(b.variant); put(b.n_class); put(b.residual); put(b.use_smem); put(b.taps_smem); put(b.hist_smem);
    put(N); put(c->n_mu); put(c->n_taps); put((uint64_t)c->tap_min); put(c->fx_bits);
    put(c->n_px); put(c->row_len); put(c->pad);
    putd(c->delta); putd(c->lam_s); putd(c->t_quiet);
    putp(out); putp(c->stream); putp(c->q32); putp(c->a32[0]); putp(c->a32[1]); putp(c->cell_I);
    putp(c->cell_bin); putp(c->cell_mu); putp(c->cell_mu32); putp(c->flags); putp(c->cell_x);
    const DevBuf* bufs[] = {&c->b_items, &c->b_regions, &c->b_phases, &c->b_phase_item, &c->b_phase_block,
                            &c->b_pblocks, &c->b_order, &c->b_cellIfx, &c->b_IB, &c->b_colj, &c->b_colw, &c->b_kq,
                            &c->b_qtoff, &c->b_qgs, &c->b_qc32, &c->b_fq, &c->b_geo, &c->b_kfix,
                            &c->b_counters, &c->b_toff, &c->b_gstart, &c->b_coefs, &c->b_ticket};
    for (const DevBuf* q : bufs) putp(q->p);
    putp(rv);
    if (rv) {
        putp(c->b_win.p); putp(c->b_ccf.tab.p); putp(c->b_ccf.tmp.p); putp(c->b_ccf.m.p);
        put(rvp.n_lines); put(rvp.n_v); put(rvp.n_chunks); put(rvp.n_wgroups); put(rvp.windowed);
        put(rvp.tile_np); put(rvp.tile_blocks); put(rvp.tile_lines); put((uint64_t)rvp.tc_chunk);
        putd(rvp.v_lo); putd(rvp.v_step); putd(rvp.h);
    }
    if (!c->b_graph_exec || c->b_graph_key != key) {
        if (c->b_graph_exec) { cudaGraphExecDestroy(c->b_graph_exec); c->b_graph_exec = nullptr; }
        c->b_graph_key.clear();
        cudaStream_t cap = nullptr;
        SOAP_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        const cudaStream_t saved = c->stream;
        const uint64_t launches0 = c->launches;
        c->stream = cap;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        soap_status st = SOAP_OK;
        cudaGraph_t graph = nullptr;
        if (e == cudaSuccess) {
            st = enqueue_batch(c, b, out, rv, &rvp);
            const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
            if (e2 != cudaSuccess && st == SOAP_OK) e = e2;
        }
        c->stream = saved;
        c->b_graph_kernels = c->launches - launches0;
        c->launches = launches0;
        if (st == SOAP_OK && e == cudaSuccess) e = cudaGraphInstantiate(&c->b_graph_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (st != SOAP_OK) { c->b_graph_exec = nullptr; return st; }
        if (e != cudaSuccess) {
            c->b_graph_exec = nullptr;
            set_error("batch graph capture failed: %s", cudaGetErrorString(e));
            return SOAP_ECUDA;
        }
        c->b_graph_key = key;
    }
    SOAP_CUDA(cudaGraphLaunch(c->b_graph_exec, c->stream));
    c->launches += c->b_graph_kernels;
    return SOAP_OK;
}

}  // namespace soap
