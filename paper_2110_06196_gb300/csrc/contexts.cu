// contexts.cu -- context windows of walks for SkipGram / CBOW training.
//
// GRAPE, Methods, "First and second-order RW-based embedding methods": the
// shallow models learn from windows of a given size sliding over the walks
// (SkipGram predicts the window from its centre, CBOW the centre from its
// window).  For row r and position i the window is
//     ctx[r][i][j]          = row[r][i - window + j]     j = 0 .. window-1
//     ctx[r][i][window + j] = row[r][i + 1 + j]          j = 0 .. window-1
// with -1 outside the row, at -1 entries (after a dead end) and around a -1
// centre.
//
// The kernel is bound by HBM writes: 2 * window int32 out per walk entry in.
// A block stages a tile of rows in shared memory and writes the tile's
// outputs as one contiguous, coalesced run (consecutive threads, consecutive
// 16-byte words).  Rows too long for a tile are served by a direct kernel that
// reads the row through the read-only path.
#include <algorithm>

#include "internal.h"

using namespace grape;

namespace {

constexpr int kCtxThreads = 256;
constexpr size_t kCtxSmemBytes = 48 * 1024;     // per block, without opt-in

__device__ __forceinline__ int ctx_value(const int* row, int L, int i, int j, int W, int centre) {
    const int pos = j < W ? i - W + j : i + 1 + (j - W);
    if (centre < 0 || pos < 0 || pos >= L) return -1;
    const int v = row[pos];
    return v >= 0 ? v : -1;
}

// n / d for 0 <= n < 2^24 and 1 <= d < 2^24: a float estimate, corrected once
// (the estimate is off by at most one in this range).
__device__ __forceinline__ int small_div(int n, int d, float inv_d) {
    int q = __float2int_rz((float)n * inv_d);
    if (q * d > n) --q;
    else if ((q + 1) * d <= n) ++q;
    return q;
}

// Tiles of R rows staged in shared memory; the tile's outputs, R * L * 2W
// contiguous int32, are written by consecutive threads in consecutive 16-byte
// words, each thread walking its four entries forward from one division.
__global__ void __launch_bounds__(kCtxThreads)
contexts_tiled_kernel(const int* __restrict__ rows, long long nrows, int L, int W, int R,
                      int* __restrict__ ctx) {
    extern __shared__ int4 smem4[];
    int* sm_rows = reinterpret_cast<int*>(smem4);
    const int width = 2 * W;
    const float inv_width = 1.0f / (float)width;
    const float inv_L = 1.0f / (float)L;
    for (long long r0 = (long long)blockIdx.x * R; r0 < nrows; r0 += (long long)gridDim.x * R) {
        const int nr = (int)(nrows - r0 < R ? nrows - r0 : R);
        const int nin = nr * L;
        const int* src = rows + r0 * L;
        for (int e = threadIdx.x; e < nin; e += blockDim.x) sm_rows[e] = __ldg(src + e);
        __syncthreads();
        const int nout = nin * width;                 // < 2^24 (R is chosen for it)
        int* dst = ctx + r0 * L * (long long)width;
        // leading entries up to a 16-byte boundary of dst, then whole words
        const int head = (int)(((16u - (reinterpret_cast<uintptr_t>(dst) & 15u)) & 15u) >> 2);
        for (int e = threadIdx.x; e < head && e < nout; e += blockDim.x) {
            const int c = small_div(e, width, inv_width);
            const int r = small_div(c, L, inv_L);
            const int i = c - r * L;
            const int* row = sm_rows + r * L;
            dst[e] = ctx_value(row, L, i, e - c * width, W, row[i]);
        }
        const int nwords = (nout - head) >> 2;
        int4* d4 = reinterpret_cast<int4*>(dst + head);
        for (int k = threadIdx.x; k < nwords; k += blockDim.x) {
            const int e = head + 4 * k;
            int c = small_div(e, width, inv_width);
            int j = e - c * width;
            int r = small_div(c, L, inv_L);
            int i = c - r * L;
            int v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int* row = sm_rows + r * L;
                v[u] = ctx_value(row, L, i, j, W, row[i]);
                if (++j == width) {
                    j = 0;
                    if (++i == L) {
                        i = 0;
                        ++r;
                    }
                }
            }
            d4[k] = make_int4(v[0], v[1], v[2], v[3]);
        }
        for (int e = head + 4 * nwords + threadIdx.x; e < nout; e += blockDim.x) {
            const int c = small_div(e, width, inv_width);
            const int r = small_div(c, L, inv_L);
            const int i = c - r * L;
            const int* row = sm_rows + r * L;
            dst[e] = ctx_value(row, L, i, e - c * width, W, row[i]);
        }
        __syncthreads();
    }
}

// One thread per (row, position) for rows whose tile does not fit.
__global__ void __launch_bounds__(kCtxThreads)
contexts_direct_kernel(const int* __restrict__ rows, long long nrows, int L, int W,
                       int* __restrict__ ctx) {
    const long long width = 2LL * W;
    const long long n = nrows * L;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const long long r = c / L;
        const int i = (int)(c - r * L);
        const int* row = rows + r * L;
        const int centre = __ldg(row + i);
        int* o = ctx + c * width;
        for (int j = 0; j < 2 * W; ++j) {
            const int pos = j < W ? i - W + j : i + 1 + (j - W);
            int v = -1;
            if (centre >= 0 && pos >= 0 && pos < L) {
                v = __ldg(row + pos);
                if (v < 0) v = -1;
            }
            o[j] = v;
        }
    }
}

}  // namespace

extern "C" {

grape_status_t grape_contexts_from_rows(const int32_t* rows, int64_t num_rows, int32_t walk_len,
                                        int32_t window, int32_t* contexts,
                                        grape_stream_t stream_) {
    if (!rows || !contexts || num_rows < 0 || walk_len < 1 || window < 1 ||
        window > GRAPE_MAX_CONTEXT_WINDOW)
        return GRAPE_ERR_INVALID_ARG;
    if (num_rows > INT64_MAX / walk_len / (2 * (int64_t)window)) return GRAPE_ERR_INVALID_ARG;
    if (num_rows == 0) return GRAPE_OK;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    int dev = 0, sms = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);
    // rows per tile: the staged rows fit the block's shared memory and the
    // tile's outputs stay below 2^24 entries (small_div's range)
    const size_t row_bytes = (size_t)walk_len * sizeof(int32_t);
    const long long out_per_row = (long long)walk_len * 2 * window;
    const long long r_smem = (long long)(kCtxSmemBytes / row_bytes);
    const long long r_out = ((1LL << 24) - 1) / out_per_row;
    const int R = (int)std::min<long long>(64, std::min(r_smem, r_out));
    if (R >= 1) {
        const size_t smem = (size_t)R * row_bytes;
        const long long tiles = (num_rows + R - 1) / R;
        const int blocks = (int)std::min<long long>(tiles, (long long)sms * 16);
        contexts_tiled_kernel<<<blocks, kCtxThreads, smem, stream>>>(rows, num_rows, walk_len,
                                                                    window, R, contexts);
    } else {
        const long long n = num_rows * (long long)walk_len;
        const int blocks = (int)std::min<long long>((n + kCtxThreads - 1) / kCtxThreads,
                                                    (long long)sms * 8);
        contexts_direct_kernel<<<blocks, kCtxThreads, 0, stream>>>(rows, num_rows, walk_len,
                                                                   window, contexts);
    }
    return cuda_status(cudaGetLastError());
}

grape_status_t grape_walk_contexts(const grape_graph_t* g, const int32_t* starts,
                                   int64_t num_starts, int32_t walk_len, int32_t walks_per_node,
                                   double p, double q, uint64_t seed, int32_t window,
                                   int64_t walk_begin, int64_t walk_count, int32_t* centres,
                                   int32_t* contexts, grape_stream_t stream_) {
    if (!g || !contexts || window < 1 || window > GRAPE_MAX_CONTEXT_WINDOW || walk_count < 0)
        return GRAPE_ERR_INVALID_ARG;
    WalkConst probe;
    grape_status_t st = make_walk_const(g, starts, num_starts, walk_len, walks_per_node, p, q,
                                        seed, contexts, &probe);
    if (st != GRAPE_OK) return st;
    st = restrict_walks(&probe, walk_begin, walk_count);
    if (st != GRAPE_OK) return st;
    if (walk_count > INT64_MAX / walk_len / (2 * (int64_t)window)) return GRAPE_ERR_INVALID_ARG;
    if (walk_count == 0) return GRAPE_OK;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    int32_t* rows = centres;
    if (!rows) {
        const cudaError_t e = cudaMallocAsync(&rows, sizeof(int32_t) * (size_t)walk_count *
                                                         (size_t)walk_len, stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    st = grape_walks_range(g, starts, num_starts, walk_len, walks_per_node, p, q, seed, walk_begin,
                           walk_count, rows, stream_);
    if (st == GRAPE_OK) st = grape_contexts_from_rows(rows, walk_count, walk_len, window, contexts,
                                                      stream_);
    if (!centres) {
        const cudaError_t e = cudaFreeAsync(rows, stream);
        if (st == GRAPE_OK && e != cudaSuccess) st = cuda_status(e);
    }
    return st;
}

}  // extern "C"
