// direct.cu -- G2: the direct form of the quiet disk sum (Alg. 1 / Alg. 4), one cell at a
// time: F_q[m] = sum_c I_c [(1 - w_c) S_b(c)[m - j_c] + w_c S_b(c)[m - j_c + 1]].
//
// The visible cells are compacted once per geometry into records {I (1 - w), I w, row offset
// b row_len - j}, ordered by (mu bin, shift phase, tap, cell index): consecutive cells then read
// the same stretch of the same row, and a warp keeps the values it loaded in registers until the
// row offset changes (every cell still adds its own two products per pixel).  k_direct: a block
// of 4 warps owns a tile of pixels and a contiguous split of the cells, staged in shared memory
// in chunks; a thread owns 4 vectors of 16 bytes of consecutive pixels (16 float or 8 double).
// For a cell, a warp's pixels read one contiguous stretch of the cell's row.  The rows are kept
// in E copies shifted by 0 .. E-1 elements (k_dir_shift, once per upload), so each thread reads
// its 4 vectors aligned from the copy whose shift matches the cell's (the same for the whole
// warp: the tile starts on a vector boundary), and the one value past its last vector -- the
// second tap of its last pixel -- is the next lane's first value, taken with __shfl_down_sync
// (lane 31, or a lane whose neighbour is past the grid, reads it itself).  FP32 sums over a chunk
// are folded into FP64 accumulators, and the splits are reduced in a fixed order by a second
// kernel, so the result is deterministic.
#include <algorithm>
#include <climits>
#include <vector>

#include "soap_internal.cuh"

namespace soap {

template <typename T>
struct DirCell {
    T I0, I1;            // I (1 - w), I w
    long long off;       // b row_len - j
};

constexpr int kDirThreads = 128;
constexpr int kDirChunk = 256;

// copies[k][e] = rows[e + k], k = 0 .. E-1 (the end value repeats past the last element).
template <typename T>
__global__ void k_dir_shift(int64_t n, int E, const T* __restrict__ rows, T* __restrict__ copies) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < E; k++) copies[(int64_t)k * n + e] = rows[e + k < n ? e + k : n - 1];
}

// 16-byte vector of T and its E elements.
template <typename T> struct Vec;
template <> struct Vec<float> {
    using V = float4;
    static constexpr int E = 4;
    __device__ static void put(const V& v, float* x) { x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w; }
    __device__ static V shfl_down(const V& v) {
        return make_float4(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1),
                           __shfl_down_sync(0xffffffffu, v.z, 1), __shfl_down_sync(0xffffffffu, v.w, 1));
    }
};
template <> struct Vec<double> {
    using V = double2;
    static constexpr int E = 2;
    __device__ static void put(const V& v, double* x) { x[0] = v.x; x[1] = v.y; }
    __device__ static V shfl_down(const V& v) {
        return make_double2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
    }
};


template <typename T>
__global__ void __launch_bounds__(kDirThreads)
k_direct(const int* __restrict__ n_cells_dev, int splits, const DirCell<T>* __restrict__ cells,
         const T* __restrict__ copies, int64_t copy_len, int64_t pad, int64_t n_px, double* __restrict__ partial) {
    using VT = Vec<T>;
    using V = typename VT::V;
    constexpr int E = VT::E;
    constexpr int NV = 4;                                  // vectors per thread
    constexpr int WPX = 32 * NV * E;                       // pixels per warp
    __shared__ DirCell<T> sc[kDirChunk];
    const int lane = threadIdx.x & 31;
    const int n_cells = *n_cells_dev;
    const int per = (n_cells + splits - 1) / splits;
    const int c_begin = (int)blockIdx.y * per;
    const int c_end = min(n_cells, c_begin + per);
    const int64_t mw = ((int64_t)blockIdx.x * (kDirThreads / 32) + (threadIdx.x >> 5)) * WPX;   // warp's first pixel
    // vector q of this lane is the warp's vector 32 q + lane: pixels mv[q] .. mv[q] + E - 1, so a
    // warp-wide load covers 32 consecutive vectors.  Vectors past the grid read the last valid one
    // (results discarded); a vector whose neighbour is past the grid, or the last vector of the
    // warp, reads its next value itself.
    const int64_t m_lastv = (n_px - 1) / E * E;
    int64_t off_v[NV];
    bool own[NV];
#pragma unroll
    for (int q = 0; q < NV; q++) {
        const int64_t mv = mw + (int64_t)(32 * q + lane) * E;
        off_v[q] = (mv <= m_lastv ? mv : m_lastv) - mw;
        own[q] = mv + E > m_lastv || (q == NV - 1 && lane == 31);
    }
    double accd[NV][E];
#pragma unroll
    for (int q = 0; q < NV; q++)
#pragma unroll
        for (int e = 0; e < E; e++) accd[q][e] = 0.0;
    // the row values of the current stretch, kept while consecutive cells read the same one
    // (cells are ordered by mu bin, shift phase and tap)
    T x[NV][E + 1];
    long long cur_off = LLONG_MIN;
    for (int cb = c_begin; cb < c_end; cb += kDirChunk) {
        __syncthreads();
        for (int t = threadIdx.x; t < kDirChunk; t += kDirThreads)
            if (cb + t < c_end) sc[t] = cells[cb + t];
        __syncthreads();
        const int nc = min(kDirChunk, c_end - cb);
        T acc[NV][E];
#pragma unroll
        for (int q = 0; q < NV; q++)
#pragma unroll
            for (int e = 0; e < E; e++) acc[q][e] = T(0);
        for (int t = 0; t < nc; t++) {
            const DirCell<T> cl = sc[t];
            if (cl.off != cur_off) {                       // warp-uniform: a new row stretch
                cur_off = cl.off;
                const int64_t e0 = cl.off + pad + mw;     // row element of the warp's first pixel
                const int r = (int)(e0 & (E - 1));
                // copy r at e0 - r holds rows[e0 ...]: aligned vectors
                const T* base = copies + (int64_t)r * copy_len + (e0 - r);
#pragma unroll
                for (int q = 0; q < NV; q++) VT::put(__ldg(reinterpret_cast<const V*>(base + off_v[q])), x[q]);
#pragma unroll
                for (int q = 0; q < NV; q++) {
                    // next value: the next lane's first, or for lane 31 lane 0's first of the next vector
                    const T down = __shfl_down_sync(0xffffffffu, x[q][0], 1);
                    const T wrap = q + 1 < NV ? __shfl_sync(0xffffffffu, x[q + 1 < NV ? q + 1 : q][0], 0) : T(0);
                    x[q][E] = lane == 31 ? wrap : down;
                    if (own[q]) x[q][E] = __ldg(base + off_v[q] + E);
                }
            }
#pragma unroll
            for (int q = 0; q < NV; q++)
#pragma unroll
                for (int e = 0; e < E; e++) acc[q][e] = fma(cl.I0, x[q][e], fma(cl.I1, x[q][e + 1], acc[q][e]));
        }
#pragma unroll
        for (int q = 0; q < NV; q++)
#pragma unroll
            for (int e = 0; e < E; e++) accd[q][e] += (double)acc[q][e];
    }
#pragma unroll
    for (int q = 0; q < NV; q++) {
        const int64_t mv = mw + (int64_t)(32 * q + lane) * E;
#pragma unroll
        for (int e = 0; e < E; e++)
            if (mv + e < n_px) partial[(int64_t)blockIdx.y * n_px + mv + e] = accd[q][e];
    }
}

template <typename T>
__global__ void k_reduce_splits(int64_t n_px, int splits, const double* __restrict__ partial, T* out) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n_px;
         m += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < splits; k++) s += partial[(int64_t)k * n_px + m];
        out[m] = (T)s;
    }
}

template <typename T>
static soap_status run_direct(soap_ctx* c, const T* rows, T* dst) {
    const int N = c->N;
    const int prec = sizeof(T) == 8 ? SOAP_FP64 : SOAP_FP32;
    constexpr int E = Vec<T>::E;
    constexpr int PX = 4 * E;                              // pixels per thread
    if (c->dir_version != c->geo_version || c->dir_prec != prec) {
        // compact the visible cells once per geometry and precision (on the host: the cell tables
        // come back once, the call synchronises its stream this one time)
        const size_t NN = (size_t)N * N;
        std::vector<double> I(NN), w(NN);
        std::vector<int32_t> jt(NN), bin(NN);
        SOAP_CUDA(cudaMemcpyAsync(I.data(), c->cell_I, NN * 8, cudaMemcpyDeviceToHost, c->stream));
        SOAP_CUDA(cudaMemcpyAsync(w.data(), c->cell_w, NN * 8, cudaMemcpyDeviceToHost, c->stream));
        SOAP_CUDA(cudaMemcpyAsync(jt.data(), c->cell_j, NN * 4, cudaMemcpyDeviceToHost, c->stream));
        SOAP_CUDA(cudaMemcpyAsync(bin.data(), c->cell_bin, NN * 4, cudaMemcpyDeviceToHost, c->stream));
        SOAP_CUDA(cudaStreamSynchronize(c->stream));
        std::vector<int32_t> idx;
        idx.reserve(NN);
        for (size_t k = 0; k < NN; k++)
            if (bin[k] >= 0) idx.push_back((int32_t)k);
        auto phase = [&](int32_t k) { return (int)(((c->pad - jt[k]) % E + E) % E); };
        std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) {
            if (bin[x] != bin[y]) return bin[x] < bin[y];
            if (phase(x) != phase(y)) return phase(x) < phase(y);
            return jt[x] < jt[y];
        });
        std::vector<DirCell<T>> rec(std::max<size_t>(1, idx.size()));
        for (size_t q = 0; q < idx.size(); q++) {
            const int32_t k = idx[q];
            rec[q].I0 = (T)(I[k] * (1.0 - w[k]));
            rec[q].I1 = (T)(I[k] * w[k]);
            rec[q].off = (long long)bin[k] * c->row_len - jt[k];
        }
        SOAP_TRY(ensure(c->dir_cells, rec.size() * sizeof(DirCell<T>)));
        SOAP_TRY(ensure(c->dir_count, sizeof(int)));
        const int n_cells = (int)idx.size();
        SOAP_CUDA(cudaMemcpyAsync(c->dir_cells.p, rec.data(), rec.size() * sizeof(DirCell<T>),
                                  cudaMemcpyHostToDevice, c->stream));
        SOAP_CUDA(cudaMemcpyAsync(c->dir_count.p, &n_cells, sizeof(int), cudaMemcpyHostToDevice, c->stream));
        SOAP_CUDA(cudaStreamSynchronize(c->stream));             // the host vectors go out of scope
        c->dir_version = c->geo_version;
        c->dir_prec = prec;
    }
    // the rows shifted by 0 .. E-1 elements, rebuilt when the rows change
    const int64_t copy_len = (int64_t)c->n_mu * c->row_len;
    if (c->dir_rows_version != c->rows_version || c->dir_rows_src != (const void*)rows) {
        SOAP_TRY(ensure(c->dir_rows, (size_t)E * copy_len * sizeof(T)));
        const int64_t g = std::min<int64_t>((copy_len + 255) / 256, 152 * 8);
        k_dir_shift<T><<<(unsigned)g, 256, 0, c->stream>>>(copy_len, E, rows, c->dir_rows.as<T>());
        SOAP_LAUNCHED(c);
        c->dir_rows_version = c->rows_version;
        c->dir_rows_src = rows;
    }
    const int64_t tiles = (c->n_px + (int64_t)kDirThreads * PX - 1) / ((int64_t)kDirThreads * PX);
    // one wave: as many splits as keep every SM's resident blocks busy; the cell count is read on
    // the device
    int dev = 0, sms = 152, per_sm = 4;
    SOAP_CUDA(cudaGetDevice(&dev));
    SOAP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SOAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_direct<T>, kDirThreads, 0));
    int64_t splits = std::max<int64_t>(1, (int64_t)sms * std::max(per_sm, 1) / tiles);
    const int64_t max_splits = ((int64_t)N * N + kDirChunk - 1) / kDirChunk;
    splits = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(splits, max_splits), 256));
    SOAP_TRY(ensure(c->partial, (size_t)splits * c->n_px * sizeof(double)));
    cudaEvent_t tb = c->profiling ? timer_begin(c) : nullptr;
    dim3 grid((unsigned)tiles, (unsigned)splits);
    k_direct<T><<<grid, kDirThreads, 0, c->stream>>>(c->dir_count.as<int>(), (int)splits,
                                                     c->dir_cells.as<DirCell<T>>(), c->dir_rows.as<T>(), copy_len,
                                                     c->pad, c->n_px, c->partial.as<double>());
    SOAP_LAUNCHED(c);
    int64_t g = (c->n_px + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    k_reduce_splits<T><<<(unsigned)g, 256, 0, c->stream>>>(c->n_px, (int)splits, c->partial.as<double>(), dst);
    SOAP_LAUNCHED(c);
    if (c->profiling) timer_end(c, SOAP_TIMER_DIRECT, tb);
    return SOAP_OK;
}

soap_status direct_quiet(soap_ctx* c, int precision, void* dst) {
    SOAP_TRY(join_geometry(c));
    if (precision == SOAP_FP64) return run_direct<double>(c, c->q64, (double*)dst);
    return run_direct<float>(c, c->q32, (float*)dst);
}

}  // namespace soap
