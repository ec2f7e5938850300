// toeplitz_tc.cu -- the Toeplitz form of the active-phase disk sum (Eqs. 1-4, Alg. 5) on the
// tensor cores (tcgen05), BF16 split precision with FP32 accumulation (SOAP_BF16X3).
//
// With K[p][cl][b][j] the per-phase velocity kernels of class cl (tap j = kernel index
// tap_min + j, exact fixed point) and the quiet group's kernel -sum_cl K (every active cell has
// exactly one owner), the three effects are
//   F[p][m] = F_q[m] + sum_(cl, b, j) K[p][cl][b][j] * X_cl,b[m][j],
//   X_cl,b[m][j] = C_cl(,b)[m] S_a(cl),b[m - k] - S_q,b[m - k]     (TOT)
//                  (C_cl(,b)[m] - 1) S_q,b[m - k]                    (FLUX)
//                  S_a(cl),b[m - k] - S_q,b[m - k]                   (BCONV),   k = tap_min + j,
// i.e. one GEMM per effect: M = pixels, N = phases, K = (class, mu bin, tap).  The contrast
// multiplies at the output pixel, so it enters X, which is built per pixel tile in shared memory
// (the Toeplitz operand: row m holds the shifted row values of every (class, bin, tap)); the
// kernel matrix K is the same for every pixel tile.
//
// Split precision: x = hi + lo with hi = bf16(x), lo = bf16(x - hi) (16 significant bits), and
// X K ~ X_hi K_hi + X_hi K_lo + X_lo K_hi, three BF16 MMAs into one FP32 accumulator.
//
// k_tc_coefs: K as BF16 hi / lo rows [phase][kk], kk = (cl n_mu + b) n_taps + j, zero-padded to
// 64-multiples; kb_nz[phase tile][K block] marks the 64 x 64 blocks with a non-zero value.
// k_toeplitz_tc: CTA = (tile of 128 pixels, tile of 64 phases, effect), 128 threads.  For each
// K block of 64 with a non-zero kernel, every thread writes its pixel's 64 operand values (hi and
// lo) into a shared stage in the 128-byte-swizzle K-major layout and copies its share of the
// kernel block; one thread issues the 12 MMAs (M = 128, N = 64, K = 16; three products) and
// commits them to the stage's barrier, so building block i+1 overlaps the MMAs of block i (two
// stages).  The epilogue reads the accumulator (lane = pixel, column = phase), adds F_q and
// stores each phase's row with 32 consecutive pixels per warp instruction.  Every barrier wait is
// bounded; a timeout sets kFlagTimeout and the CTA stops issuing work.
#include <cuda_bf16.h>

#include "soap_internal.cuh"
#include "tc_gemm.cuh"

namespace soap {

constexpr int kTcM = 128;                 // pixels per CTA (TMEM lanes)
constexpr int kTcN = 128;                 // phases per CTA (accumulator columns)
constexpr int kTcK = 64;                  // K per block: one 128-byte swizzle row of BF16
constexpr int kTcThreads = 256;           // two threads per operand row
constexpr int kTcAB = kTcM * kTcK * 2;    // bytes of one operand-tile half (hi or lo), 16 KB
constexpr int kTcBB = kTcN * kTcK * 2;    // bytes of one kernel-tile half, 16 KB
constexpr int kTcStage = 2 * kTcAB + 2 * kTcBB;
constexpr int kTcStages = 2;

// Byte offset of 16-byte chunk c (elements 8c .. 8c+7) of row r in a 128-byte-swizzle K-major
// tile: rows of 128 bytes, the chunk index XORed with the row's place in its group of 8 rows.
__device__ __forceinline__ uint32_t sw128(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// hi = bf16(x), lo = bf16(x - hi) for two values, packed as two bf16x2 words
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hw, uint32_t& lw) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    hw = *reinterpret_cast<const uint32_t*>(&h);
    lw = *reinterpret_cast<const uint32_t*>(&l);
}

// K[p][kk] (fixed point, [n_phases][k_tot] as k_phase_hist leaves it) -> BF16 hi / lo rows of
// k_pad columns for p < p_pad; marks the non-zero (128 phases x 64) blocks.
__global__ void k_tc_coefs(const long long* __restrict__ kfix, int n_phases, int k_tot, int p_pad, int k_pad,
                           int fx_bits, __nv_bfloat16* __restrict__ khi, __nv_bfloat16* __restrict__ klo,
                           unsigned int* __restrict__ kb_nz) {
    const int n_kb = k_pad / kTcK;
    const int64_t total = (int64_t)p_pad * k_pad;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(i / k_pad), kk = (int)(i - (int64_t)p * k_pad);
        const long long K = (p < n_phases && kk < k_tot) ? kfix[(int64_t)p * k_tot + kk] : 0;
        const float x = fixed_to_float(K, fx_bits);
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        khi[i] = hi;
        klo[i] = __float2bfloat16_rn(x - __bfloat162float(hi));
        if (K != 0) atomicOr(&kb_nz[(p / kTcN) * n_kb + kk / kTcK], 1u);
    }
}

struct TcArgs {
    int64_t n_px;
    int64_t row_len, pad;
    int tap_min, n_taps, n_mu, ncl, k_tot, k_pad, n_phases;
    int win;                          // staged row window: kTcM + n_taps - 1, rounded up to 4
    int n_crow;                       // contrast rows: ncl, or ncl n_mu (per bin)
    int per_bin;
    const float* rows[3];             // quiet, spot, facula rows [n_mu][row_len]
    int type[SOAP_MAX_CLASSES];       // region type of each class
    const float* con;                 // contrast rows [n_crow][n_px]
    const float* fq;                  // quiet integral [n_px]
    const __nv_bfloat16* khi;         // kernel rows [p_pad][k_pad]
    const __nv_bfloat16* klo;
    const unsigned int* kb_nz;        // [p_pad / 128][k_pad / 64]
};

// Shared memory after the operand ring: row windows [3][n_mu][win] and one zero window,
// contrast [n_crow][kTcM], decode table [k_pad] (int4: quiet-row, active-row and contrast offsets),
// non-zero flags of the K blocks, barriers.
__host__ __device__ inline size_t tc_smem_bytes(int n_mu, int win, int n_crow, int k_pad) {
    return (size_t)kTcStages * kTcStage + 1024 + ((size_t)3 * n_mu + 1) * win * 4 + (size_t)n_crow * kTcM * 4 +
           (size_t)k_pad * 16 + ((size_t)k_pad / kTcK * 4 + 7) / 8 * 8 + 64;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int EFF>
__global__ void __launch_bounds__(kTcThreads, 1)
k_toeplitz_tc(const __grid_constant__ TcArgs g, float* __restrict__ out, unsigned int* flags) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* ring = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int set_len = g.n_mu * g.win;
    const int n_kb = g.k_pad / kTcK;
    float* s_rows = reinterpret_cast<float*>(ring + kTcStages * kTcStage);
    float* s_con = s_rows + 3 * set_len + g.win;                     // after the zero window
    int4* s_tab = reinterpret_cast<int4*>(s_con + g.n_crow * kTcM);
    int* s_nz = reinterpret_cast<int*>(s_tab + g.k_pad);
    uint64_t* empty = reinterpret_cast<uint64_t*>(s_nz + (n_kb + 1) / 2 * 2);
    uint64_t* accum = empty + kTcStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    const int t = threadIdx.x, warp = t >> 5;
    const int r = t & (kTcM - 1), half = t / kTcM;  // operand row (pixel) and which 32 of its 64 values
    const int64_t m0 = (int64_t)blockIdx.x * kTcM;
    const int pt = blockIdx.y, p0 = pt * kTcN;

    if (t == 0) {
        for (int s = 0; s < kTcStages; s++) tc::mbar_init(&empty[s], 1);
        tc::mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(tc::smem_u32(tmem_slot)), "r"(kTcN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // row windows (asynchronous copies): s_rows[set][b][i] = rows_set,b[m0 - tap_min - (n_taps - 1) + i]
    // for i < kTcM + n_taps - 1 (every tap of every pixel of the tile), zero beyond and in the zero
    // window; two rows at a time, thread r copying elements r and r + kTcM
    const int wlen = kTcM + g.n_taps - 1;
    for (int row = half; row < 3 * g.n_mu; row += 2) {
        const int set = row / g.n_mu, b = row - set * g.n_mu;
        const float* src = (set == 0 ? g.rows[0] : (set == 1 ? g.rows[1] : g.rows[2])) + (int64_t)b * g.row_len +
                           g.pad + m0 - g.tap_min - (g.n_taps - 1);
        for (int i = r; i < g.win; i += kTcM) {
            if (i < wlen) cp_async4(s_rows + row * g.win + i, src + i);
            else s_rows[row * g.win + i] = 0.0f;
        }
    }
    for (int i = t; i < g.win; i += kTcThreads) s_rows[3 * set_len + i] = 0.0f;
    if (EFF != SOAP_EFFECT_BCONV)
        for (int idx = t; idx < g.n_crow * kTcM; idx += kTcThreads) {
            const int cr = idx / kTcM;
            const int64_t mm = m0 + (idx - cr * kTcM);
            cp_async4(s_con + idx, g.con + (int64_t)cr * g.n_px + (mm < g.n_px ? mm : g.n_px - 1));
        }
    // decode table (while the copies run): kk = (cl n_mu + b) n_taps + j -> offsets of the quiet
    // and active row values of tap j in bin b and of the contrast row; padding -> the zero window
    for (int kk = t; kk < g.k_pad; kk += kTcThreads) {
        const int per_class = g.n_mu * g.n_taps;
        const int cl = kk / per_class, rem = kk - cl * per_class;
        const int b = rem / g.n_taps, j = rem - b * g.n_taps;
        int4 e = make_int4(3 * set_len, 3 * set_len, 0, 0);
        if (cl < g.ncl) {
            const int off = b * g.win + (g.n_taps - 1 - j);
            const int set = g.type[cl] == SOAP_FACULA ? 2 : 1;
            e = make_int4(off, set * set_len + off, (g.per_bin ? cl * g.n_mu + b : cl) * kTcM, 0);
        }
        s_tab[kk] = e;
    }
    for (int kb = t; kb < n_kb; kb += kTcThreads) s_nz[kb] = g.kb_nz[pt * n_kb + kb] != 0;
    cp_async_wait_all();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    int it = 0;                                     // K blocks issued
    bool ok = true;
    for (int kb = 0; kb < n_kb; kb++) {
        if (!s_nz[kb]) continue;                    // all kernels of this block are zero
        const int s = it & 1;
        if (it >= kTcStages) ok = tc::mbar_wait(&empty[s], ((it - kTcStages) / kTcStages) & 1, flags);
        if (!__syncthreads_and(ok)) { ok = false; break; }
        unsigned char* st = ring + s * kTcStage;
        // kernel rows p0 .. p0+127 of this block (hi and lo: 2048 chunks of 16 bytes, 8 per thread),
        // copied asynchronously while the operand is built
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int idx = 8 * t + q;
            const int row = idx >> 4, hl = (idx >> 3) & 1, c = idx & 7;
            cp_async16(st + 2 * kTcAB + hl * kTcBB + sw128(row, c),
                       (hl ? g.klo : g.khi) + (int64_t)(p0 + row) * g.k_pad + (int64_t)kb * kTcK + 8 * c);
        }
        // this thread's 32 operand values of row r (kk = kb 64 + 32 half + 0 .. 31), 8 per chunk
#pragma unroll 1
        for (int q = 0; q < 4; q++) {
            const int c8 = 4 * half + q;
            const int kk0 = kb * kTcK + 8 * c8;
            float x[8];
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const int4 te = s_tab[kk0 + e];
                const float rq = s_rows[te.x + r];
                if (EFF == SOAP_EFFECT_BCONV) x[e] = s_rows[te.y + r] - rq;
                else if (EFF == SOAP_EFFECT_FLUX) x[e] = (s_con[te.z + r] - 1.0f) * rq;
                else x[e] = fmaf(s_con[te.z + r], s_rows[te.y + r], -rq);
            }
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int e = 0; e < 4; e++) split2(x[2 * e], x[2 * e + 1], hw[e], lw[e]);
            *reinterpret_cast<uint4*>(st + sw128(r, c8)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(st + kTcAB + sw128(r, c8)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        cp_async_wait_all();
        // the tensor cores read shared memory through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = tc::smem_u32(st), al = ah + kTcAB, bh = al + kTcAB, bl = bh + kTcBB;
            constexpr uint32_t idesc = tc::idesc_bf16(kTcN);
#pragma unroll
            for (int k = 0; k < kTcK / 16; k++) {
                tc::mma_bf16(tmem, tc::sdesc(ah + k * 32), tc::sdesc(bh + k * 32), idesc, (it | k) != 0);
                tc::mma_bf16(tmem, tc::sdesc(ah + k * 32), tc::sdesc(bl + k * 32), idesc, 1u);
                tc::mma_bf16(tmem, tc::sdesc(al + k * 32), tc::sdesc(bh + k * 32), idesc, 1u);
            }
            tc::mma_commit(&empty[s]);
        }
        it++;
    }

    // accumulator complete (every MMA issued above has finished) before it is read or released
    if (t == 0 && it > 0) tc::mma_commit(accum);
    bool done = ok;
    if (it > 0) done = tc::mbar_wait(accum, 0, flags) && done;
    done = __syncthreads_and(done);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (done) {
        // warp w: TMEM lanes 32 (w & 3) .. +31 (its pixels), columns 64 (w >> 2) .. +63 (its phases)
        const int lg = warp & 3;
        const int64_t me = m0 + 32 * lg + (t & 31);
        const float f0 = g.fq[me < g.n_px ? me : g.n_px - 1];
#pragma unroll 1
        for (int c = 64 * (warp >> 2); c < 64 * (warp >> 2) + 64; c += 32) {
            if (p0 + c >= g.n_phases) break;
            float v[32];
            if (it > 0) {
                tc::tmem_ld32(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)c, v);
            } else {
#pragma unroll
                for (int i = 0; i < 32; i++) v[i] = 0.0f;
            }
            if (me < g.n_px) {
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    const int p = p0 + c + i;
                    if (p < g.n_phases) out[(int64_t)p * g.n_px + me] = f0 + v[i];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN) : "memory");
    }
}

soap_status toeplitz_tc(soap_ctx* c, const long long* kfix, int n_phases, int ncl, const int* class_type,
                        const float* a_spot, const float* a_fac, const float* con32, bool per_bin,
                        const int* effects, int n_eff, float* out) {
    const int k_tot = ncl * c->n_mu * c->n_taps;
    const int k_pad = (k_tot + kTcK - 1) / kTcK * kTcK;
    const int p_pad = (n_phases + kTcN - 1) / kTcN * kTcN;
    const int n_kb = k_pad / kTcK;
    const int win = (kTcM + c->n_taps - 1 + 3) / 4 * 4;
    const int n_crow = per_bin ? ncl * c->n_mu : ncl;
    const size_t smem = tc_smem_bytes(c->n_mu, win, n_crow, k_pad);
    if (smem > 227 * 1024) {
        set_error("SOAP_BF16X3 needs %zu bytes of shared memory per block for %d mu bins, %d taps and %d classes "
                  "(at most %d)", smem, c->n_mu, c->n_taps, ncl, 227 * 1024);
        return SOAP_ERANGE;
    }
    const size_t kb_bytes = (size_t)p_pad * k_pad * sizeof(__nv_bfloat16);
    const size_t off_lo = (kb_bytes + 255) / 256 * 256;
    const size_t off_nz = off_lo + (kb_bytes + 255) / 256 * 256;
    const size_t nz_bytes = (size_t)(p_pad / kTcN) * n_kb * sizeof(unsigned int);
    SOAP_TRY(ensure(c->tc_coef, off_nz + nz_bytes));
    __nv_bfloat16* khi = c->tc_coef.as<__nv_bfloat16>();
    __nv_bfloat16* klo = reinterpret_cast<__nv_bfloat16*>(c->tc_coef.as<char>() + off_lo);
    unsigned int* nz = reinterpret_cast<unsigned int*>(c->tc_coef.as<char>() + off_nz);
    SOAP_CUDA(cudaMemsetAsync(nz, 0, nz_bytes, c->stream));
    const int64_t total = (int64_t)p_pad * k_pad;
    const int cg = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8));
    k_tc_coefs<<<cg, 256, 0, c->stream>>>(kfix, n_phases, k_tot, p_pad, k_pad, c->fx_bits, khi, klo, nz);
    SOAP_LAUNCHED(c);

    TcArgs g{};
    g.n_px = c->n_px;
    g.row_len = c->row_len;
    g.pad = c->pad;
    g.tap_min = c->tap_min;
    g.n_taps = c->n_taps;
    g.n_mu = c->n_mu;
    g.ncl = ncl;
    g.k_tot = k_tot;
    g.k_pad = k_pad;
    g.n_phases = n_phases;
    g.win = win;
    g.n_crow = n_crow;
    g.per_bin = per_bin ? 1 : 0;
    g.rows[0] = c->q32;
    g.rows[1] = a_spot;
    g.rows[2] = a_fac;
    for (int k = 0; k < ncl && k < SOAP_MAX_CLASSES; k++) g.type[k] = class_type ? class_type[k] : SOAP_SPOT;
    g.con = con32;
    g.fq = c->fq.as<float>();
    g.khi = khi;
    g.klo = klo;
    g.kb_nz = nz;
    dim3 grid((unsigned)((c->n_px + kTcM - 1) / kTcM), (unsigned)(p_pad / kTcN));
    for (int e = 0; e < n_eff; e++) {
        float* oe = out + (int64_t)e * n_phases * c->n_px;
        auto launch = [&](auto kern) -> soap_status {
            SOAP_TRY(fit_dynamic_smem(kern, smem));
            SOAP_TIMED(c, SOAP_TIMER_CONTRACT,
                       kern<<<grid, kTcThreads, smem, c->stream>>>(g, oe, c->flags);
                       SOAP_LAUNCHED(c));
            return SOAP_OK;
        };
        if (effects[e] == SOAP_EFFECT_FLUX) SOAP_TRY(launch(k_toeplitz_tc<SOAP_EFFECT_FLUX>));
        else if (effects[e] == SOAP_EFFECT_BCONV) SOAP_TRY(launch(k_toeplitz_tc<SOAP_EFFECT_BCONV>));
        else SOAP_TRY(launch(k_toeplitz_tc<SOAP_EFFECT_TOT>));
    }
    return SOAP_OK;
}

}  // namespace soap
