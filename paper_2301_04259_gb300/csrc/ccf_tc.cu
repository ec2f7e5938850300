// ccf_tc.cu -- the line-mask CCF of Sect. 4.1 on the tensor cores (tcgen05), BF16 split
// precision with FP32 accumulation (SOAP_BF16X3 calls and soap_rv_ccf with spectra_f32 = 2).
//
// With A_lk = U_l + f_l + S_k + g_k the start of line l's box at velocity k (pixel n covers
// [n, n+1) in these coordinates, as in ccf.cu), the CCF is one matrix product
//   CCF[s][k] = sum_n F[s][n] M[k][n],   M[k][n] = sum_l w_l |[n, n+1) intersect [A_lk, A_lk + box)|,
// with M = spectra, N = velocities and K = pixels.
//
// k_ccf_tc_m builds the mask matrix once per mask and velocity grid (it is kept with the line
// tables): one CTA per 64-pixel K block, one thread per (velocity, 32-pixel half row), which
// adds the overlaps of the few lines that reach those pixels (staged in shared memory) in a
// private FP32 row and stores it split, x = hi + lo with hi = bf16(x), lo = bf16(x - hi), as the
// 128-byte-swizzle K-major image of the block's shared-memory tile (hi tile, then lo tile).
// k_ccf_tc: CTA = (chunk of pixels, tile of 128 spectra), one CTA per SM, warp-specialised (see
// the kernel): one lane streams the mask tiles of each K block with a bulk copy into a ring of up
// to four stages, another copies the block's FP32 spectra into the A stage with a TMA tensor copy
// (16-byte aligned rows; otherwise they are loaded into registers), eight warps split them in
// place into the BF16 hi/lo tiles, one lane issues the 12 MMAs of the block (M = 128, N = velocities
// rounded up to 16, K = 16; F_hi M_hi + F_hi M_lo + F_lo M_hi) once both stages are full and
// commits them to the barriers that free the stages.  The epilogue writes the chunk's FP32
// partial CCF, which k_ccf_reduce adds over the chunks in a fixed order.  Every barrier wait is
// bounded; a timeout sets kFlagTimeout and the CTA stops issuing work.
#include <cuda_bf16.h>
#include <climits>

#include "soap_internal.cuh"
#include "tc_gemm.cuh"

namespace soap {

constexpr int kCcM = 128;                  // spectra per CTA (TMEM lanes)
constexpr int kCcK = 64;                   // pixels per K block: one 128-byte swizzle row of BF16
constexpr int kCcThreads = 256;            // mask-matrix builder threads
constexpr int kCcChunkMax = 2048;          // pixels per CTA at most (bounds the FP32 accumulation)
// mask-matrix builder
constexpr int kCcWin = 512;                // lines of a K block staged in shared memory (more: read directly)
constexpr int kCcMaxV = 256;               // velocities at most (N <= 256)

__host__ __device__ inline int cc_bb(int n_pad) { return n_pad * kCcK * 2; }       // one mask-tile half
__host__ __device__ inline size_t cc_m_smem() {
    return (size_t)kCcThreads * 32 * 4 + (size_t)kCcWin * 12 + (size_t)kCcMaxV * 8;
}

__device__ __forceinline__ void cc_split2(float x0, float x1, uint32_t& hw, uint32_t& lw) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    hw = *reinterpret_cast<const uint32_t*>(&h);
    lw = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ uint32_t cc_sw128(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// first line l in [0, n) with U[l] >= key (U non-decreasing)
__device__ __forceinline__ int cc_lower(const int* __restrict__ U, int n, int64_t key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int64_t)__ldg(U + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// the 8 values x[0..7] as one 16-byte chunk of hi and one of lo (shared or global memory)
__device__ __forceinline__ void cc_put8(unsigned char* hi_tile, unsigned char* lo_tile, uint32_t off,
                                        const float* x) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int e = 0; e < 4; e++) cc_split2(x[2 * e], x[2 * e + 1], hw[e], lw[e]);
    *reinterpret_cast<uint4*>(hi_tile + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

struct CcMArgs {
    const int* U;          // [n_lines] integer part of each line's box start (sorted, non-decreasing)
    const float* f;        // [n_lines] fraction of the box start, [0, 1)
    const int* valid;      // [n_lines] 0: the box leaves the grid somewhere on the velocity grid
    const float* w;        // [n_lines] line weights
    const int* S;          // [n_v] integer part of the velocity shift atanh(v/c)/Delta
    const float* g;        // [n_v] its fraction, [0, 1)
    unsigned char* m;      // [n_kb][hi, lo][n_pad x 128 bytes]
    int n_lines, n_v, n_pad;
    int lo_off;            // lines with U < p - lo_off cannot reach pixel p at any velocity
    int hi_off;            // lines with U >= p + hi_off cannot reach pixels below p + kCcK
    float box;
};

__global__ void __launch_bounds__(kCcThreads)
k_ccf_tc_m(const __grid_constant__ CcMArgs g) {
    extern __shared__ __align__(16) unsigned char cc_m_raw[];
    float* scratch = reinterpret_cast<float*>(cc_m_raw);                  // element j of thread t at j * 256 + t
    int* sLU = reinterpret_cast<int*>(scratch + kCcThreads * 32);
    float* sLF = reinterpret_cast<float*>(sLU + kCcWin);
    float* sLW = sLF + kCcWin;
    int* sS = reinterpret_cast<int*>(sLW + kCcWin);
    float* sG = reinterpret_cast<float*>(sS + kCcMaxV);
    const int t = threadIdx.x;
    const int64_t p = (int64_t)blockIdx.x * kCcK;
    const int la = cc_lower(g.U, g.n_lines, p - g.lo_off);
    const int lb = max(la, cc_lower(g.U, g.n_lines, p + g.hi_off));
    const int nl = lb - la;
    for (int i = t; i < min(nl, kCcWin); i += kCcThreads) {
        const int l = la + i;
        sLU[i] = __ldg(g.U + l);
        sLF[i] = __ldg(g.f + l);
        sLW[i] = __ldg(g.valid + l) ? __ldg(g.w + l) : 0.0f;       // lines whose box leaves the grid: skipped
    }
    for (int k = t; k < g.n_v; k += kCcThreads) {
        sS[k] = __ldg(g.S + k);
        sG[k] = __ldg(g.g + k);
    }
    __syncthreads();
    unsigned char* hi = g.m + (size_t)blockIdx.x * 2 * cc_bb(g.n_pad);
    unsigned char* lo = hi + cc_bb(g.n_pad);
    float* my = scratch + t;
    for (int task = t; task < 2 * g.n_pad; task += kCcThreads) {
        const int k = task >> 1, hb = task & 1;
        const int64_t q0 = p + 32 * hb;
#pragma unroll
        for (int j = 0; j < 32; j++) my[j * kCcThreads] = 0.0f;
        if (k < g.n_v) {
            const int Sk = sS[k];
            const float gk = sG[k];
            for (int i = 0; i < nl; i++) {
                int Ul;
                float fl, wl;
                if (i < kCcWin) {
                    Ul = sLU[i]; fl = sLF[i]; wl = sLW[i];
                } else {                                    // a dense stretch of the mask
                    const int l = la + i;
                    Ul = __ldg(g.U + l); fl = __ldg(g.f + l);
                    wl = __ldg(g.valid + l) ? __ldg(g.w + l) : 0.0f;
                }
                // the box starts at base + xf in the pixel units of this row half
                const int base = (int)((int64_t)Ul + Sk - q0);
                if (base >= 32) break;                      // so do those of all later lines
                if (wl == 0.0f) continue;
                const float xf = fl + gk;                   // in [0, 2)
                int j = base + (xf >= 1.0f ? 1 : 0);        // pixel holding the box start
                if (j < 0) j = 0;
                for (; j < 32; j++) {
                    const float av = xf - (float)(j - base);       // box start relative to pixel j
                    if (av + g.box <= 0.0f) break;                 // the box ended before pixel j
                    my[j * kCcThreads] += wl * (fminf(av + g.box, 1.0f) - fmaxf(av, 0.0f));
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float x[8];
#pragma unroll
            for (int e = 0; e < 8; e++) x[e] = my[(8 * q + e) * kCcThreads];
            cc_put8(hi, lo, cc_sw128(k, 4 * hb + q), x);
        }
    }
}

struct CcArgs {
    const unsigned char* m;   // mask tiles from k_ccf_tc_m
    const float* spectra;     // [n_spec][n_px] FP32
    float* partial;           // [n_chunks][n_spec][n_v] FP32
    int64_t n_px;
    int64_t chunk;            // pixels per chunk (a multiple of kCcK)
    int n_v, n_pad, n_spec;
    int vec4;                 // rows are 16-byte aligned: 16-byte loads
    int ra;                   // spectrum rows an A stage holds (a multiple of 8, at most 128)
    uint32_t tmem_cols;
};


// 32 spectrum values of row frow at pixels pa .. pa+31, zero at and past P1 (or for no row)
__device__ __forceinline__ void cc_load_row(float (&a)[32], const float* frow, bool row_on, int vec4,
                                            int64_t pa, int64_t P1) {
    if (row_on && vec4 && pa + 32 <= P1) {
        const float4* src = reinterpret_cast<const float4*>(frow + pa);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const float4 v = __ldg(src + q);
            a[4 * q] = v.x; a[4 * q + 1] = v.y; a[4 * q + 2] = v.z; a[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int e = 0; e < 32; e++) a[e] = (row_on && pa + e < P1) ? __ldg(frow + pa + e) : 0.0f;
    }
}

// Warp-specialised form.  Warp 0, one lane: the mask tiles of K block kb, one bulk copy of both
// halves into B stage kb mod SB (completion on fullB, transaction bytes).  Warps 2..9 (256
// threads): the spectrum values of block kb split into the A stage kb mod SA, after which each
// thread fences its writes for the tensor cores and arrives on fullA.  Warp 1, one lane: when both
// stages are full, the 12 MMAs of the block, committed to emptyA and emptyB, which free the
// stages for the copies and splits of later blocks.  So the tensor cores, the copies and the
// splits of different K blocks overlap, the mask tiles SB - 1 blocks ahead of the MMAs.
// The splitters take the spectrum values from one of two places:
//  - TMA (16-byte aligned rows): warp 10, one lane, copies the FP32 block (128 rows x 64 px, rows
//    past the last spectrum and pixels past the grid read as zero) into the A stage itself once
//    the MMAs have released it (fullR); the splitters read it back (lanes along the pixels of two
//    rows per warp access), agree on a named barrier that every value was read, and overwrite the
//    stage with its BF16 hi/lo tiles.  No spectrum value passes through the load queues.
//  - registers (any alignment): two threads per spectrum row load the row's values of block kb + 1
//    while block kb is split, and write block kb once the MMAs have released its stage.
constexpr int kCcWsThreads = 352;
// A (spectra) stages: three when they are filled by TMA; two when the splitters load the values
// through L1 themselves (the smaller ring leaves more of the SM's memory to L1)
__host__ __device__ constexpr int cc_sa(bool tma) { return tma ? 3 : 2; }
constexpr int kCcSAMax = 3;
constexpr int kCcSBMax = 4;                // B (mask) stages at most
// An A stage holds ra rows (the spectra of the largest tile rounded up to 8, at most 128): the
// hi tile's rows at 128 r, then the lo tile's at ra x 128 + 128 r.  The MMAs read 128 rows of
// each; the rows from ra on hold other data (the lo tile, the next stage, the mask ring) and
// only reach accumulator lanes of spectra the tile does not have, which are never read.
__host__ __device__ inline int cc_ab(int ra) { return ra * kCcK * 2; }         // one half (hi or lo)
__host__ __device__ inline int cc_sb(int n_pad, int ra, int sa) {
    const long avail = 227L * 1024 - 1024 - 256 - (long)sa * 2 * cc_ab(ra);
    const long sb = avail / (2L * cc_bb(n_pad));
    return (int)(sb < kCcSBMax ? sb : kCcSBMax);
}
// the epilogue's transpose tiles (32 x 33 floats per warp, eight warps) reuse the rings
constexpr int kCcEpi = 8 * 32 * 33 * 4;
__host__ __device__ inline size_t cc_rings(int n_pad, int ra, int sa) {
    const size_t r = (size_t)sa * 2 * cc_ab(ra) + (size_t)cc_sb(n_pad, ra, sa) * 2 * cc_bb(n_pad);
    return r > (size_t)kCcEpi ? r : (size_t)kCcEpi;
}
__host__ __device__ inline size_t cc_ws_smem(int n_pad, int ra, int sa) { return cc_rings(n_pad, ra, sa) + 1024 + 256; }

__device__ __forceinline__ void cc_mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cc_bulk(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(tc::smem_u32(dst)), "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
                 : "memory");
}
// named barrier 1 over the 256 splitter threads: true when v holds in every one of them
__device__ __forceinline__ bool cc_split_all(bool v) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbarrier.red.and.pred q, 1, 256, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r) : "r"((uint32_t)v) : "memory");
    return r != 0;
}

template <bool kTmaA>
__global__ void __launch_bounds__(kCcWsThreads, 1)
k_ccf_tc(const __grid_constant__ CcArgs g, const __grid_constant__ CUtensorMap map_f, unsigned int* flags) {
    extern __shared__ unsigned char smem_raw[];
    // the reduction after this kernel may launch now: it waits for this grid before reading
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    unsigned char* base = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int bb = cc_bb(g.n_pad);
    const int ab = cc_ab(g.ra);
    constexpr int SA = cc_sa(kTmaA);
    const int SB = cc_sb(g.n_pad, g.ra, SA);
    unsigned char* ringA = base;                                   // [SA][hi, lo][ra x 128 B]
    unsigned char* ringB = ringA + SA * 2 * ab;                    // [SB][hi, lo][n_pad x 128 B]
    uint64_t* fullA = reinterpret_cast<uint64_t*>(base + cc_rings(g.n_pad, g.ra, SA));
    uint64_t* emptyA = fullA + kCcSAMax;
    uint64_t* fullR = emptyA + kCcSAMax;
    uint64_t* fullB = fullR + kCcSAMax;
    uint64_t* emptyB = fullB + kCcSBMax;
    uint64_t* accum = emptyB + kCcSBMax;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int64_t P0 = (int64_t)blockIdx.x * g.chunk;
    const int64_t P1 = P0 + g.chunk < g.n_px ? P0 + g.chunk : g.n_px;
    const int n_kb = (int)((P1 - P0 + kCcK - 1) / kCcK);
    const int64_t kb0 = P0 / kCcK;                  // first K block of the chunk in the mask tiles
    const int s0 = blockIdx.y * kCcM;

    if (t == 0) {
        for (int s = 0; s < SA; s++) {
            tc::mbar_init(&fullA[s], 256);
            tc::mbar_init(&emptyA[s], 1);
            tc::mbar_init(&fullR[s], 1);
        }
        for (int s = 0; s < SB; s++) { tc::mbar_init(&fullB[s], 1); tc::mbar_init(&emptyB[s], 1); }
        tc::mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(tc::smem_u32(tmem_slot)), "r"(g.tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // producer: mask tiles, SB - 1 blocks ahead of the MMAs
            int armed = 0;
            for (int kb = 0; kb < n_kb; kb++) {
                const int s = kb % SB;
                if (!tc::mbar_wait(&emptyB[s], ((kb / SB) & 1) ^ 1, flags)) break;
                tc::mbar_expect_tx(&fullB[s], 2u * (uint32_t)bb);
                cc_bulk(ringB + (size_t)s * 2 * bb, g.m + (size_t)(kb0 + kb) * 2 * bb, 2u * (uint32_t)bb, &fullB[s]);
                armed = kb + 1;
            }
            // the last copies issued must land before the CTA may exit
            for (int kb = armed - 1; kb >= 0 && kb >= armed - SB; kb--)
                tc::mbar_wait(&fullB[kb % SB], (kb / SB) & 1, flags);
        }
    } else if (warp == 10) {
        if (kTmaA && lane == 0) {
            // producer: FP32 spectrum blocks (ra rows) into the A stages the MMAs have released,
            // once the kernel that wrote them has finished (a no-op without an early start)
            asm volatile("griddepcontrol.wait;" ::: "memory");
            int armed = 0;
            for (int kb = 0; kb < n_kb; kb++) {
                const int s = kb % SA;
                if (!tc::mbar_wait(&emptyA[s], ((kb / SA) & 1) ^ 1, flags)) break;
                tc::mbar_expect_tx(&fullR[s], 2u * (uint32_t)ab);
                tc::tma_load_2d(ringA + (size_t)s * 2 * ab, &map_f, (int)(P0 + (int64_t)kb * kCcK), s0, &fullR[s]);
                armed = kb + 1;
            }
            for (int kb = armed - 1; kb >= 0 && kb >= armed - SA; kb--)
                tc::mbar_wait(&fullR[kb % SA], (kb / SA) & 1, flags);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            const uint32_t idesc = tc::idesc_bf16(g.n_pad);
            for (int kb = 0; kb < n_kb; kb++) {
                const int sa = kb % SA, sb = kb % SB;
                if (!tc::mbar_wait(&fullA[sa], (kb / SA) & 1, flags)) break;
                if (!tc::mbar_wait(&fullB[sb], (kb / SB) & 1, flags)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ah = tc::smem_u32(ringA + (size_t)sa * 2 * ab), al = ah + (uint32_t)ab;
                const uint32_t bh = tc::smem_u32(ringB + (size_t)sb * 2 * bb), bl = bh + (uint32_t)bb;
#pragma unroll
                for (int k = 0; k < kCcK / 16; k++) {
                    tc::mma_bf16(tmem, tc::sdesc(ah + k * 32), tc::sdesc(bh + k * 32), idesc, (kb | k) != 0);
                    tc::mma_bf16(tmem, tc::sdesc(ah + k * 32), tc::sdesc(bl + k * 32), idesc, 1u);
                    tc::mma_bf16(tmem, tc::sdesc(al + k * 32), tc::sdesc(bh + k * 32), idesc, 1u);
                }
                tc::mma_commit(&emptyA[sa]);
                tc::mma_commit(&emptyB[sb]);
            }
            tc::mma_commit(accum);          // arrives once every MMA issued above has completed
        }
    } else if (kTmaA) {
        // splitters on the staged block: warp w' = warp - 2 takes rows 16 w' .. 16 w' + 15, two
        // rows per access (lanes 0-15 and 16-31), four pixels per lane
        const int w8 = warp - 2, j = lane & 15;
        for (int kb = 0; kb < n_kb; kb++) {
            const int sa = kb % SA;
            const bool ok = tc::mbar_wait(&fullR[sa], (kb / SA) & 1, flags);
            unsigned char* st = ringA + (size_t)sa * 2 * ab;
            float4 v[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const int r = 16 * w8 + 2 * i + (lane >> 4);
                if (r < g.ra) v[i] = *reinterpret_cast<const float4*>(st + r * (kCcK * 4) + j * 16);
            }
            if (!cc_split_all(ok)) break;                  // every value of the stage read (or a wait gave up)
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const int r = 16 * w8 + 2 * i + (lane >> 4);
                if (r >= g.ra) continue;
                uint2 hw, lw;
                cc_split2(v[i].x, v[i].y, hw.x, lw.x);
                cc_split2(v[i].z, v[i].w, hw.y, lw.y);
                const uint32_t off = cc_sw128(r, j >> 1) + (uint32_t)(j & 1) * 8;
                *reinterpret_cast<uint2*>(st + off) = hw;
                *reinterpret_cast<uint2*>(st + ab + off) = lw;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");     // visible to the tensor cores
            cc_mbar_arrive(&fullA[sa]);
        }
    } else {
        // splitters from registers: spectrum row r, pixels 32 h .. 32 h + 31 of each K block
        const int u = t - 64;
        const int r = u & (kCcM - 1), half = u >> 7;
        const bool row_on = s0 + r < g.n_spec;
        const float* frow = g.spectra + (int64_t)(row_on ? s0 + r : 0) * g.n_px;
        asm volatile("griddepcontrol.wait;" ::: "memory");     // the spectra's writer has finished
        float a[32], a1[32];
        cc_load_row(a, frow, row_on, g.vec4, P0 + 32 * half, P1);
        auto split = [&](int kb, float (&cur)[32], float (&nxt)[32]) -> bool {
            if (kb + 1 < n_kb) cc_load_row(nxt, frow, row_on, g.vec4, P0 + (int64_t)(kb + 1) * kCcK + 32 * half, P1);
            const int sa = kb % SA;
            if (!tc::mbar_wait(&emptyA[sa], ((kb / SA) & 1) ^ 1, flags)) return false;
            unsigned char* st = ringA + (size_t)sa * 2 * ab;
            if (r < g.ra) {
#pragma unroll
                for (int q = 0; q < 4; q++) cc_put8(st, st + ab, cc_sw128(r, 4 * half + q), cur + 8 * q);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");     // visible to the tensor cores
            cc_mbar_arrive(&fullA[sa]);
            return true;
        };
        for (int kb = 0; kb < n_kb; kb += 2) {
            if (!split(kb, a, a1)) break;
            if (kb + 1 < n_kb && !split(kb + 1, a1, a)) break;
        }
    }

    // accumulator complete before it is read or released (every MMA issued has finished)
    const bool epi = warp >= 2 && warp < 10;
    bool done = true;
    if (epi) done = __all_sync(0xffffffffu, tc::mbar_wait(accum, 0, flags));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (epi && done) {
        // warp w: TMEM lanes 32 (w & 3) .. +31 (its spectra), column blocks of 32 alternating
        // between the two groups of four warps (its velocities); each 32 x 32 block goes out
        // through the warp's shared tile (every MMA has completed, so the rings are free), one
        // spectrum's 32 velocities per store
        const int lg = warp & 3;
        const int grp = (warp - 2) >> 2;
        float (*tile)[33] = reinterpret_cast<float (*)[33]>(base + (size_t)(warp - 2) * 32 * 33 * 4);
        float* dst = g.partial + (int64_t)blockIdx.x * g.n_spec * g.n_v;
#pragma unroll 1
        for (int c = 32 * grp; c < g.n_pad; c += 64) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)c, v);
            tc::store_rows(tile, v, lane, dst, g.n_v, s0 + 32 * lg, g.n_spec, c, g.n_v);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols) : "memory");
    }
}

bool ccf_tc_fits(int n_v) {
    const int n_pad = (n_v + 15) / 16 * 16;
    for (int sa = 2; sa <= kCcSAMax; sa++)
        if (cc_sb(n_pad, kCcM, sa) < 2 || cc_ws_smem(n_pad, kCcM, sa) > 227 * 1024) return false;
    return n_v >= 1 && n_v <= kCcMaxV;
}

int64_t ccf_tc_chunk(int64_t n_px, int n_spec, int sms) {
    const int64_t tiles = (n_spec + kCcM - 1) / kCcM;
    const int64_t per = (n_px * tiles + sms - 1) / std::max(sms, 1);     // pixels per CTA for one wave
    const int64_t chunk = (per + kCcK - 1) / kCcK * kCcK;
    return std::max<int64_t>(kCcK, std::min<int64_t>(chunk, kCcChunkMax));
}

soap_status ccf_tc_build_m(soap_ctx* c, CcfState& st, const CcfPlan& p) {
    // the mask matrix of this mask and velocity grid (kept until either changes)
    const int n_pad = (p.n_v + 15) / 16 * 16;
    const int64_t n_kb = (c->n_px + kCcK - 1) / kCcK;
    const double box = 2.0 * p.h;
    SOAP_TRY(ensure(st.m, (size_t)n_kb * 2 * cc_bb(n_pad)));
    CcMArgs m{};
    m.U = p.U;
    m.f = p.f32t;
    m.valid = p.valid;
    m.w = p.w32;
    m.S = p.S;
    m.g = p.g32;
    m.m = st.m.as<unsigned char>();
    m.n_lines = p.n_lines;
    m.n_v = p.n_v;
    m.n_pad = n_pad;
    // a line reaches pixels [p, p + 64) at velocity k only if U + S_k < p + 64 and
    // U + S_k + 2 + box > p (box start U + S_k + f + g with f + g < 2); S_min, S_max carry a margin
    m.lo_off = p.tc_smax + 2 + (int)std::ceil(box) + 1;
    m.hi_off = kCcK - p.tc_smin + 1;
    m.box = (float)box;
    SOAP_TRY(fit_dynamic_smem(k_ccf_tc_m, cc_m_smem()));
    k_ccf_tc_m<<<(unsigned)n_kb, kCcThreads, cc_m_smem(), c->stream>>>(m);
    SOAP_LAUNCHED(c);
    st.m_ok = true;
    st.m_fresh = true;
    return SOAP_OK;
}

soap_status ccf_tc(soap_ctx* c, CcfState& st, const CcfPlan& p, const float* spectra, float* partial) {
    const int n_pad = (p.n_v + 15) / 16 * 16;
    CcArgs a{};
    a.m = st.m.as<unsigned char>();
    a.spectra = spectra;
    a.partial = partial;
    a.n_px = c->n_px;
    a.chunk = p.tc_chunk;
    a.n_v = p.n_v;
    a.n_pad = n_pad;
    a.n_spec = p.n_spec;
    a.vec4 = (reinterpret_cast<uintptr_t>(spectra) % 16 == 0 && c->n_px % 4 == 0) ? 1 : 0;
    uint32_t cols = 32;
    while ((int)cols < n_pad) cols <<= 1;
    a.tmem_cols = cols;
    a.ra = (int)std::min<int64_t>(kCcM, ((int64_t)p.n_spec + 7) / 8 * 8);
    dim3 grid((unsigned)((c->n_px + p.tc_chunk - 1) / p.tc_chunk), (unsigned)((p.n_spec + kCcM - 1) / kCcM));
    // Programmatic dependent launch: the CTAs may start while the kernel queued before this one
    // finishes (it lets them go once all its CTAs have started), set up their barriers and TMEM
    // and stream the first mask tiles; whatever reads the spectra waits for that kernel first
    // (griddepcontrol.wait).  Not when that kernel wrote the mask matrix itself.
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = st.m_fresh ? 0 : 1;
    st.m_fresh = false;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kCcWsThreads);
    cfg.stream = c->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CUtensorMap map_f{};
    if (a.vec4 && c->n_px < INT_MAX && p.n_spec < INT_MAX) {
        // spectra [n_spec][n_px] FP32, boxes of ra rows x 64 pixels
        const uint64_t dims[2] = {(uint64_t)c->n_px, (uint64_t)p.n_spec};
        const uint64_t strides[1] = {(uint64_t)c->n_px * 4};
        const uint32_t box[2] = {(uint32_t)kCcK, (uint32_t)a.ra};
        SOAP_TRY(tc::encode_map(&map_f, 2, spectra, dims, strides, box, CU_TENSOR_MAP_DATA_TYPE_FLOAT32));
        cfg.dynamicSmemBytes = cc_ws_smem(n_pad, a.ra, cc_sa(true));
        SOAP_TRY(fit_dynamic_smem(k_ccf_tc<true>, cfg.dynamicSmemBytes));
        SOAP_CUDA(cudaLaunchKernelEx(&cfg, k_ccf_tc<true>, a, map_f, c->flags));
    } else {
        cfg.dynamicSmemBytes = cc_ws_smem(n_pad, a.ra, cc_sa(false));
        SOAP_TRY(fit_dynamic_smem(k_ccf_tc<false>, cfg.dynamicSmemBytes));
        SOAP_CUDA(cudaLaunchKernelEx(&cfg, k_ccf_tc<false>, a, map_f, c->flags));
    }
    SOAP_LAUNCHED(c);
    return SOAP_OK;
}

}  // namespace soap
