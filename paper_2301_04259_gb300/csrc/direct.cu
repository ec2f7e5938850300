// direct.cu -- G2: the direct form of the quiet disk sum (Alg. 1 / Alg. 4), one cell at a
// time: F_q[m] = sum_c I_c [(1 - w_c) S_b(c)[m - j_c] + w_c S_b(c)[m - j_c + 1]].
//
// Each block owns a tile of pixels and a contiguous split of the cells; cells are staged in
// shared memory in chunks (weights I(1-w), I w and the row offset b*row_len - j), and every
// thread walks the chunk for its pixels with coalesced loads from the replicate-padded rows.
// FP32 partial sums over a chunk are folded into FP64 accumulators; the splits are reduced
// in a fixed order by a second kernel, so the result is deterministic.
#include "soap_internal.cuh"

namespace soap {

template <typename T, int R, int THREADS, int CHUNK>
__global__ void __launch_bounds__(THREADS)
k_direct(int64_t NN, int64_t cells_per_split, const double* __restrict__ cell_I,
         const double* __restrict__ cell_w, const int32_t* __restrict__ cell_j,
         const int32_t* __restrict__ cell_bin, const T* __restrict__ rows, int64_t row_len,
         int64_t pad, int64_t n_px, double* __restrict__ partial) {
    __shared__ T sI0[CHUNK];
    __shared__ T sI1[CHUNK];
    __shared__ int64_t sOff[CHUNK];
    const int64_t c_begin = (int64_t)blockIdx.y * cells_per_split;
    const int64_t c_end = min(NN, c_begin + cells_per_split);
    const int64_t mbase = (int64_t)blockIdx.x * THREADS * R + threadIdx.x;
    int64_t mc[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        int64_t m = mbase + (int64_t)r * THREADS;
        mc[r] = pad + (m < n_px ? m : n_px - 1);
    }
    double accd[R];
#pragma unroll
    for (int r = 0; r < R; r++) accd[r] = 0.0;
    for (int64_t cb = c_begin; cb < c_end; cb += CHUNK) {
        __syncthreads();
        for (int t = threadIdx.x; t < CHUNK; t += THREADS) {
            int64_t c = cb + t;
            int b = c < c_end ? cell_bin[c] : -1;
            if (b >= 0) {
                double I = cell_I[c], w = cell_w[c];
                sI0[t] = (T)(I * (1.0 - w));
                sI1[t] = (T)(I * w);
                sOff[t] = (int64_t)b * row_len - cell_j[c];
            } else {
                sI0[t] = T(0); sI1[t] = T(0); sOff[t] = 0;
            }
        }
        __syncthreads();
        T acc[R];
#pragma unroll
        for (int r = 0; r < R; r++) acc[r] = T(0);
        const int64_t left = c_end - cb;
        const int nc = left < CHUNK ? (int)left : CHUNK;
        for (int t = 0; t < nc; t++) {
            const T a0 = sI0[t], a1 = sI1[t];
            const T* row = rows + sOff[t];
#pragma unroll
            for (int r = 0; r < R; r++)
                acc[r] = fma(a0, __ldg(row + mc[r]), fma(a1, __ldg(row + mc[r] + 1), acc[r]));
        }
#pragma unroll
        for (int r = 0; r < R; r++) accd[r] += (double)acc[r];
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
        int64_t m = mbase + (int64_t)r * THREADS;
        if (m < n_px) partial[(int64_t)blockIdx.y * n_px + m] = accd[r];
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

template <typename T, int R, int THREADS, int CHUNK>
static soap_status run_direct(soap_ctx* c, const T* rows, T* dst) {
    const int64_t NN = (int64_t)c->N * c->N;
    const int64_t tiles = (c->n_px + (int64_t)THREADS * R - 1) / ((int64_t)THREADS * R);
    int64_t splits = (4 * 152 + tiles - 1) / tiles;
    int64_t max_splits = (NN + CHUNK - 1) / CHUNK;
    if (splits > max_splits) splits = max_splits;
    if (splits > 256) splits = 256;
    if (splits < 1) splits = 1;
    int64_t per = (NN + splits - 1) / splits;
    per = (per + CHUNK - 1) / CHUNK * CHUNK;
    splits = (NN + per - 1) / per;
    SOAP_TRY(ensure(c->partial, (size_t)splits * c->n_px * sizeof(double)));
    cudaEvent_t tb = c->profiling ? timer_begin(c) : nullptr;
    dim3 grid((unsigned)tiles, (unsigned)splits);
    k_direct<T, R, THREADS, CHUNK><<<grid, THREADS, 0, c->stream>>>(
        NN, per, c->cell_I, c->cell_w, c->cell_j, c->cell_bin, rows, c->row_len, c->pad, c->n_px,
        c->partial.as<double>());
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
    if (precision == SOAP_FP64) return run_direct<double, 2, 256, 128>(c, c->q64, (double*)dst);
    return run_direct<float, 4, 256, 128>(c, c->q32, (float*)dst);
}

}  // namespace soap
