// toeplitz_tma.cu -- the Toeplitz form of the active-phase disk sum (Eqs. 1-4, Alg. 5) on the
// tensor cores (tcgen05), with the shifted operand read straight from TMA-loaded windows
// (SOAP_BF16X3; region classes with one contrast row each).
//
// On the log grid the spectrum of one phase is
//   TOT (Eq. 3):   F[m] = F_q[m] - (Q * S_q)[m] + sum_cl C_cl[m] (K_cl * S_a(cl))[m]
//   BCONV (Eq. 2): F[m] = F_q[m] - (Q * S_q)[m] + sum_cl (K_cl * S_a(cl))[m]
//   FLUX (Eq. 1):  F[m] = F_q[m] + sum_cl (C_cl[m] - 1) (K_cl * S_q)[m]
// with (K * S)[m] = sum_(b, j) K[b][j] S_b[m - tap_min - j] the convolution over mu bin b and tap j
// with the phase's velocity kernels (exact fixed point), Q = sum_cl K_cl (every active cell has
// one owner) and C_cl the Planck contrast of class cl at the output pixel (Sect. 4.3.1).  Each
// convolution is a GEMM with M = 128 output pixels (tensor-memory lanes), N = a group of NG phases
// (accumulator columns) and K = (bin, tap).  Q and every class get an accumulator of their own, so
// the contrast stays out of the operands and multiplies when the accumulators are read back.
//
// Operand A is never built.  The rows S_b are kept as BF16 hi / lo planes: plane c holds bins
// 8c .. 8c+7 of every pixel as one 16-byte row.  One TMA box per row set and hi / lo brings a
// window of W >= 127 + n_taps pixels of every plane into shared memory, rows 16 bytes apart.  In
// the canonical K-major layout without swizzle (core matrix = 8 rows of 16 bytes, 8-row groups
// SBO apart, the two K halves of an MMA LBO apart) the operand of tap j for the 128 pixels is the
// window from row W0 - j on, with SBO = 128 bytes; and with LBO = 16 bytes the second K half is
// the next row, which is the operand of tap j - 1.  So one MMA (K = 16) covers the 8 bins of a
// plane at taps 2t+1 and 2t, and a tap is only a descriptor start address.
//
// Operand B (the kernels of the group's phases for one accumulator and one K step, hi and lo)
// is built by k_tm_coefs in the matching layout (8-phase groups 128 bytes apart, K halves NG x 16
// bytes apart), with a flag per tile when any value is non-zero; the CTA streams the non-zero
// tiles through a ring with bulk copies.  Split precision as in toeplitz_tc.cu: x = hi + lo,
// X K ~ X_hi K_hi + X_hi K_lo + X_lo K_hi in FP32.
//
// CTA = 128 pixels x NG phases, 192 threads: warp 0 allocates the tensor memory and one of its
// lanes issues the copies, one lane of warp 1 issues the MMAs, warps 2-5 read the accumulators
// (lane = pixel) and store each phase's row.  Every wait is bounded (about a second of clocks); a
// wait that gives up sets kFlagTimeout, the CTA stops issuing work, waits (bounded) for what it
// issued and frees its tensor memory.
#include <cuda_bf16.h>

#include <algorithm>

#include "soap_internal.cuh"
#include "tc_gemm.cuh"

namespace soap {

constexpr int kTmM = 128;                         // pixels per CTA (TMEM lanes)
constexpr int kTmThreads = 192;
constexpr int kTmStages = 8;                      // coefficient-tile ring
constexpr int kTmMaxAcc = SOAP_MAX_CLASSES + 1;   // Q and every class
constexpr int kTmMaxTapsPad = 128;                // window of 127 + taps pixels in one TMA box (<= 256)

struct TmArgs {
    int64_t n_px;
    int64_t n_lo0;                // padded-row index of window row 0 for the tile at pixel 0
    int n_phases, NG, n_groups, n_acc, NC, W, TP, n_steps;   // TP tap pairs, n_steps = NC TP
    int eff;
    int rs_load[3];               // row sets (quiet, spot, facula) whose windows the CTA loads
    int acc_rs[kTmMaxAcc];        // row set each accumulator reads
    int acc_con[kTmMaxAcc];       // contrast row of each accumulator (class); -1 for Q
    const unsigned char* coef;    // [group][acc][step][hi, lo][NG x 32 bytes]
    const unsigned int* nz;       // [group][acc][step]
    const float* con;             // [ncl][n_px]
    const float* fq;              // [n_px]
    uint32_t tmem_cols;
};

__device__ __forceinline__ void tm_split8(const float (&x)[8], uint4& hi, uint4& lo) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * e], x[2 * e + 1]);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x[2 * e] - hf.x, x[2 * e + 1] - hf.y);
        hw[e] = *reinterpret_cast<const uint32_t*>(&h);
        lw[e] = *reinterpret_cast<const uint32_t*>(&l);
    }
    hi = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    lo = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// BF16 hi / lo planes of the FP32 padded rows: planes[(2 rs + h) NC + c][n] = bins 8c .. 8c+7 of
// row set rs at padded index n (zero past n_mu).  Grid (pixels, NC, row sets).
__global__ void k_tm_planes(int64_t row_len, int n_mu, int NC, const float* __restrict__ q,
                            const float* __restrict__ sp, const float* __restrict__ fa, uint4* __restrict__ planes) {
    const int c = blockIdx.y, rs = blockIdx.z;
    const float* rows = rs == 0 ? q : (rs == 1 ? sp : fa);
    if (!rows) return;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < row_len;
         n += (int64_t)gridDim.x * blockDim.x) {
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int b = 8 * c + e;
            x[e] = b < n_mu ? __ldg(rows + (int64_t)b * row_len + n) : 0.0f;
        }
        uint4 hi, lo;
        tm_split8(x, hi, lo);
        planes[((int64_t)(2 * rs) * NC + c) * row_len + n] = hi;
        planes[((int64_t)(2 * rs + 1) * NC + c) * row_len + n] = lo;
    }
}

// Operand B tiles.  Block = (group, accumulator, K step); thread = (K half kh, phase q of the
// group), 2 NG threads.  K step = (plane c, tap pair t): half 0 holds bins 8c .. 8c+7 at tap
// 2t+1, half 1 the same bins at tap 2t (the order of the A descriptor).  Accumulator a is Q
// (quiet_acc = 1, a = 0: the sum of the class kernels) or class a - quiet_acc.
__global__ void k_tm_coefs(const long long* __restrict__ kfix, int n_phases, int ncl, int n_mu, int n_taps,
                           int fx_bits, int NG, int n_acc, int n_steps, int TP, int quiet_acc,
                           unsigned char* __restrict__ coef, unsigned int* __restrict__ nz) {
    const int blk = blockIdx.x;                       // (group n_acc + a) n_steps + step
    const int step = blk % n_steps;
    const int a = (blk / n_steps) % n_acc;
    const int grp = blk / (n_steps * n_acc);
    const int c = step / TP, tp = step - c * TP;
    const int kh = threadIdx.x / NG, q = threadIdx.x - kh * NG;
    const int j = kh == 0 ? 2 * tp + 1 : 2 * tp;
    const int p = grp * NG + q;
    const int64_t per_cl = (int64_t)n_mu * n_taps;
    float x[8];
    bool any = false;
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const int b = 8 * c + e;
        long long K = 0;
        if (p < n_phases && b < n_mu && j < n_taps) {
            const long long* kp = kfix + (int64_t)p * ncl * per_cl + (int64_t)b * n_taps + j;
            if (quiet_acc && a == 0) {
                for (int cl = 0; cl < ncl; cl++) K += kp[cl * per_cl];
            } else {
                K = kp[(a - quiet_acc) * per_cl];
            }
        }
        any |= K != 0;
        x[e] = fixed_to_float(K, fx_bits);
    }
    uint4 hi, lo;
    tm_split8(x, hi, lo);
    const int TB = NG * 32;
    unsigned char* tile = coef + (int64_t)blk * 2 * TB;
    const int off = kh * NG * 16 + (q >> 3) * 128 + (q & 7) * 16;
    *reinterpret_cast<uint4*>(tile + off) = hi;
    *reinterpret_cast<uint4*>(tile + TB + off) = lo;
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) nz[blk] = any ? 1u : 0u;
}

// Shared-memory descriptor, K-major without swizzle: start, K-half offset (LBO) and 8-row-group
// offset (SBO) in bytes, descriptor version 1.
__device__ __forceinline__ uint64_t tm_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void tm_tma_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(tc::smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
          "r"(tc::smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tm_bulk(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(tc::smem_u32(dst)), "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tm_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

struct TmSmem {
    int box_bytes, TB;
    size_t a_off, ring_off, bar_off, nz_off, total;
    __host__ __device__ TmSmem(int NC, int W, int NG, int nsa) {
        box_bytes = NC * W * 16;
        TB = NG * 32;
        a_off = 0;
        ring_off = a_off + 6 * (size_t)box_bytes;
        bar_off = ring_off + (size_t)kTmStages * 2 * TB;
        nz_off = bar_off + (size_t)(2 * kTmStages + 2) * 8 + 8;   // barriers, tensor-memory slot
        total = 1024 + nz_off + (size_t)nsa + kTmMaxAcc + 16;      // 1024: alignment slack
    }
};

__global__ void __launch_bounds__(kTmThreads, 1)
k_toeplitz_tma(const __grid_constant__ CUtensorMap planes, const __grid_constant__ TmArgs g,
               float* __restrict__ out, unsigned int* flags) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int nsa = g.n_acc * g.n_steps;
    const TmSmem L(g.NC, g.W, g.NG, nsa);
    unsigned char* abox = base + L.a_off;                 // 6 windows: (row set, hi / lo)
    unsigned char* ring = base + L.ring_off;
    uint64_t* fullA = reinterpret_cast<uint64_t*>(base + L.bar_off);
    uint64_t* full = fullA + 1;
    uint64_t* empty = full + kTmStages;
    uint64_t* accum = empty + kTmStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    unsigned char* snz = base + L.nz_off;                 // [acc][step] non-zero tile
    unsigned char* swr = snz + nsa;                       // [acc] written by at least one MMA
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int grp = (int)(blockIdx.x % (unsigned)g.n_groups);
    const int64_t m0 = (int64_t)(blockIdx.x / (unsigned)g.n_groups) * kTmM;
    const int p0 = grp * g.NG;

    if (t == 0) {
        tc::mbar_init(fullA, 1);
        for (int s = 0; s < kTmStages; s++) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
        tc::mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = t; i < nsa; i += kTmThreads) snz[i] = g.nz[(int64_t)grp * nsa + i] != 0u ? 1 : 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(tc::smem_u32(tmem_slot)), "r"(g.tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    if (t < g.n_acc) {
        unsigned char w = 0;
        for (int s = 0; s < g.n_steps; s++) w |= snz[t * g.n_steps + s];
        swr[t] = w;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int TB = L.TB;

    if (warp == 0 && lane == 0) {
        // producer: the row windows of this pixel tile, then the non-zero coefficient tiles
        uint32_t bytes = 0;
        for (int r = 0; r < 3; r++)
            if (g.rs_load[r]) bytes += 2u * (uint32_t)L.box_bytes;
        tc::mbar_expect_tx(fullA, bytes);
        const int nlo = (int)(g.n_lo0 + m0);
        for (int r = 0; r < 3; r++)
            if (g.rs_load[r])
                for (int h = 0; h < 2; h++) tm_tma_4d(abox + (2 * r + h) * L.box_bytes, &planes, 0, nlo, 0, 2 * r + h, fullA);
        int it = 0;
        for (int i = 0; i < nsa; i++) {
            if (!snz[i]) continue;
            const int s = it % kTmStages;
            if (!tc::mbar_wait(&empty[s], ((it / kTmStages) & 1) ^ 1, flags)) break;
            tc::mbar_expect_tx(&full[s], 2u * (uint32_t)TB);
            tm_bulk(ring + s * 2 * TB, g.coef + ((int64_t)grp * nsa + i) * 2 * TB, 2u * (uint32_t)TB, &full[s]);
            it++;
        }
        // every copy issued here lands before the CTA may exit
        tc::mbar_wait(fullA, 0, flags);
        for (int k = it - 1; k >= 0 && k >= it - kTmStages; k--)
            tc::mbar_wait(&full[k % kTmStages], (k / kTmStages) & 1, flags);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = tc::idesc_bf16(g.NG);
        bool ok = tc::mbar_wait(fullA, 0, flags);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t abase = tc::smem_u32(abox), rbase = tc::smem_u32(ring);
        uint32_t started = 0;                           // bit a: accumulator a holds a sum
        int it = 0;
        for (int i = 0; i < nsa && ok; i++) {
            if (!snz[i]) continue;
            const int s = it % kTmStages;
            if (!tc::mbar_wait(&full[s], (it / kTmStages) & 1, flags)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int a = i / g.n_steps, step = i - a * g.n_steps;
            const int c = step / g.TP, tp = step - c * g.TP;
            const int i0 = 2 * g.TP - 2 - 2 * tp;        // window row of tap 2 tp + 1 at pixel 0
            const uint32_t pa = abase + (uint32_t)(2 * g.acc_rs[a] * L.box_bytes + (c * g.W + i0) * 16);
            const uint64_t ahi = tm_desc(pa, 16, 128);
            const uint64_t alo = tm_desc(pa + (uint32_t)L.box_bytes, 16, 128);
            const uint32_t pb = rbase + (uint32_t)(s * 2 * TB);
            const uint64_t bhi = tm_desc(pb, (uint32_t)g.NG * 16, 128);
            const uint64_t blo = tm_desc(pb + (uint32_t)TB, (uint32_t)g.NG * 16, 128);
            const uint32_t d = tmem + (uint32_t)(a * g.NG);
            tc::mma_bf16(d, ahi, bhi, idesc, (started >> a) & 1u);
            tc::mma_bf16(d, ahi, blo, idesc, 1u);
            tc::mma_bf16(d, alo, bhi, idesc, 1u);
            started |= 1u << a;
            tc::mma_commit(&empty[s]);
            it++;
        }
        tc::mma_commit(accum);          // arrives once every MMA issued above has completed
        tc::mbar_wait(accum, 0, flags); // (bounded) before the tensor memory can be released
    } else if (warp >= 2) {
        // epilogue: TMEM lanes 32 (warp % 4) .. +31, one pixel per lane
        const int qd = warp & 3;
        const int64_t m = m0 + 32 * qd + lane;
        const int64_t mc = m < g.n_px ? m : g.n_px - 1;
        const bool done = __all_sync(0xffffffffu, tc::mbar_wait(accum, 0, flags));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (done) {
            const float f0 = g.fq[mc];
            float cf[kTmMaxAcc];
#pragma unroll
            for (int a = 0; a < kTmMaxAcc; a++) {
                float w = 0.0f;
                if (a < g.n_acc) {
                    const int cr = g.acc_con[a];
                    if (cr < 0) w = -1.0f;                                   // Q: the quiet rows leave
                    else if (g.eff == SOAP_EFFECT_BCONV) w = 1.0f;
                    else if (g.eff == SOAP_EFFECT_FLUX) w = g.con[(int64_t)cr * g.n_px + mc] - 1.0f;
                    else w = g.con[(int64_t)cr * g.n_px + mc];
                }
                cf[a] = w;
            }
#pragma unroll 1
            for (int cc = 0; cc < g.NG; cc += 16) {
                if (p0 + cc >= g.n_phases) break;
                float v[16];
#pragma unroll
                for (int i = 0; i < 16; i++) v[i] = 0.0f;
#pragma unroll
                for (int a = 0; a < kTmMaxAcc; a++) {
                    if (a >= g.n_acc || !swr[a]) continue;               // warp-uniform
                    float x[16];
                    tm_ld16(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(a * g.NG + cc), x);
#pragma unroll
                    for (int i = 0; i < 16; i++) v[i] = fmaf(cf[a], x[i], v[i]);
                }
                if (m < g.n_px) {
#pragma unroll
                    for (int i = 0; i < 16; i++) {
                        const int p = p0 + cc + i;
                        if (p < g.n_phases) out[(int64_t)p * g.n_px + m] = f0 + v[i];
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
struct TmShape {
    int n_taps_pad, TP, NC, W, n_steps;
};

static TmShape tm_shape(const soap_ctx* c) {
    TmShape s;
    s.n_taps_pad = (c->n_taps + 1) / 2 * 2;
    s.TP = s.n_taps_pad / 2;
    s.NC = (c->n_mu + 7) / 8;
    s.W = (127 + s.n_taps_pad + 7) / 8 * 8;
    s.n_steps = s.NC * s.TP;
    return s;
}

// Phases per CTA: as many as keep the accumulators within 256 tensor-memory columns (two CTAs
// per SM), at most 64.
static int tm_group(int n_acc) {
    for (int ng = 64; ng >= 16; ng -= 16)
        if (n_acc * ng <= 256) return ng;
    return 16;
}

bool toeplitz_tma_fits(const soap_ctx* c, int ncl) {
    const TmShape s = tm_shape(c);
    const int n_acc = ncl + 1;
    if (ncl < 1 || n_acc > kTmMaxAcc || s.n_taps_pad > kTmMaxTapsPad || s.W > 256 || s.NC > 8) return false;
    const TmSmem L(s.NC, s.W, tm_group(n_acc), n_acc * s.n_steps);
    return L.total <= 227 * 1024;
}

soap_status toeplitz_tma(soap_ctx* c, const long long* kfix, int n_phases, int ncl, const int* class_type,
                         const float* a_spot, const float* a_fac, const float* con32, const int* effects, int n_eff,
                         float* out) {
    if (!toeplitz_tma_fits(c, ncl)) { set_error("shape outside the TMA contraction's limits"); return SOAP_ERANGE; }
    const TmShape s = tm_shape(c);
    // BF16 planes of the rows, rebuilt when the rows or the active row sets changed
    const size_t plane_bytes = (size_t)6 * s.NC * (size_t)c->row_len * 16;
    if (c->tm_planes_version != c->rows_version || c->tm_planes_src[0] != c->q32 || c->tm_planes_src[1] != a_spot ||
        c->tm_planes_src[2] != a_fac || c->tm_planes.bytes < plane_bytes) {
        SOAP_TRY(ensure(c->tm_planes, plane_bytes));
        dim3 grid((unsigned)std::min<int64_t>((c->row_len + 255) / 256, 152 * 4), (unsigned)s.NC, 3);
        k_tm_planes<<<grid, 256, 0, c->stream>>>(c->row_len, c->n_mu, s.NC, c->q32, a_spot, a_fac,
                                                 c->tm_planes.as<uint4>());
        SOAP_LAUNCHED(c);
        c->tm_planes_version = c->rows_version;
        c->tm_planes_src[0] = c->q32;
        c->tm_planes_src[1] = a_spot;
        c->tm_planes_src[2] = a_fac;
    }
    CUtensorMap map;
    {
        const uint64_t dims[4] = {8, (uint64_t)c->row_len, (uint64_t)s.NC, 6};
        const uint64_t strides[3] = {16, (uint64_t)c->row_len * 16, (uint64_t)s.NC * c->row_len * 16};
        const uint32_t box[4] = {8, (uint32_t)s.W, (uint32_t)s.NC, 1};
        SOAP_TRY(tc::encode_map(&map, 4, c->tm_planes.p, dims, strides, box));
    }
    bool need_flux = false, need_tot = false;
    for (int e = 0; e < n_eff; e++) {
        if (effects[e] == SOAP_EFFECT_FLUX) need_flux = true;
        else need_tot = true;
    }
    const int n_tiles = (int)((c->n_px + kTmM - 1) / kTmM);
    // coefficient tiles: one set for TOT / BCONV (Q and the classes), one for FLUX (classes), in
    // one buffer sized for both before anything is launched
    const int NG = tm_group(ncl + 1);
    const int n_groups = (n_phases + NG - 1) / NG;
    const int TB = NG * 32;
    size_t off[2][2] = {{0, 0}, {0, 0}};          // [pass][tiles, flags]
    size_t total = 0;
    for (int pass = 0; pass < 2; pass++) {
        const size_t nblk = (size_t)n_groups * (ncl + (pass == 0 ? 1 : 0)) * s.n_steps;
        off[pass][0] = total;
        total += (nblk * 2 * TB + 255) / 256 * 256;
        off[pass][1] = total;
        total += (nblk * 4 + 255) / 256 * 256;
    }
    SOAP_TRY(ensure(c->tm_coef, total));
    for (int pass = 0; pass < 2; pass++) {
        const bool flux = pass == 1;
        if ((flux && !need_flux) || (!flux && !need_tot)) continue;
        const int quiet_acc = flux ? 0 : 1;
        const int n_acc = ncl + quiet_acc;
        const size_t nblk = (size_t)n_groups * n_acc * s.n_steps;
        unsigned char* coef = c->tm_coef.as<unsigned char>() + off[pass][0];
        unsigned int* nz = reinterpret_cast<unsigned int*>(c->tm_coef.as<unsigned char>() + off[pass][1]);
        k_tm_coefs<<<(unsigned)nblk, 2 * NG, 0, c->stream>>>(kfix, n_phases, ncl, c->n_mu, c->n_taps, c->fx_bits, NG,
                                                             n_acc, s.n_steps, s.TP, quiet_acc, coef, nz);
        SOAP_LAUNCHED(c);
        TmArgs g{};
        g.n_px = c->n_px;
        g.n_lo0 = c->pad - c->tap_min - (s.n_taps_pad - 1);
        g.n_phases = n_phases;
        g.NG = NG;
        g.n_groups = n_groups;
        g.n_acc = n_acc;
        g.NC = s.NC;
        g.W = s.W;
        g.TP = s.TP;
        g.n_steps = s.n_steps;
        g.coef = coef;
        g.nz = nz;
        g.con = con32;
        g.fq = c->fq.as<float>();
        uint32_t cols = 32;
        while ((int)cols < n_acc * NG) cols <<= 1;
        g.tmem_cols = cols;
        for (int a = 0; a < n_acc; a++) {
            const int cl = a - quiet_acc;
            const int type = cl >= 0 ? class_type[cl] : 0;
            g.acc_rs[a] = (cl < 0 || flux) ? 0 : (type == SOAP_FACULA ? 2 : 1);
            g.acc_con[a] = cl;
            g.rs_load[g.acc_rs[a]] = 1;
        }
        const TmSmem L(s.NC, s.W, NG, n_acc * s.n_steps);
        SOAP_TRY(fit_dynamic_smem(k_toeplitz_tma, L.total));
        for (int e = 0; e < n_eff; e++) {
            if ((effects[e] == SOAP_EFFECT_FLUX) != flux) continue;
            g.eff = effects[e];
            float* oe = out + (int64_t)e * n_phases * c->n_px;
            SOAP_TIMED(c, SOAP_TIMER_CONTRACT,
                       k_toeplitz_tma<<<(unsigned)((int64_t)n_tiles * n_groups), kTmThreads, L.total, c->stream>>>(
                           map, g, oe, c->flags);
                       SOAP_LAUNCHED(c));
        }
    }
    return SOAP_OK;
}

}  // namespace soap
