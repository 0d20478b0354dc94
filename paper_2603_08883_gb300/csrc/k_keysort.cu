// Direct stable LSD radix sort of the rows in canonical order, for export.
//
// The rows are split into columns (x words, z words, the coefficient's bits)
// and every pass moves whole columns: per tile of 2048 elements a histogram of
// one 8-bit digit, a multi-block exclusive scan over (digit, tile), and a
// stable scatter whose ranks come from warp-local counters (each warp owns 256
// consecutive elements; lanes with the same digit find each other with
// match_any) and whose writes are staged in shared memory in digit order, so
// no key is ever gathered through a permutation and writes leave in runs.  Digits that
// are constant over all elements are skipped.  Canonical order compares x as
// an integer with its last word most significant, then z likewise, so the
// passes run over z_0, ..., z_{Wd-1}, then x_0, ..., x_{Wd-1}, low byte first.
#include <cuda_runtime.h>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;
constexpr int kBins = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxCols = 9;  // 2 Wd + 1 for Wd = 4

struct Cols {
    uint64_t* c[kMaxCols];
};

__global__ void k_rows_to_cols(const uint64_t* __restrict__ rows, const double* __restrict__ coef, int stride,
                               int64_t n, Cols out) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        for (int w = 0; w < stride; ++w) out.c[w][i] = rows[i * stride + w];
        out.c[stride][i] = (uint64_t)__double_as_longlong(coef[i]);
    }
}

// OR and AND of every key column (orand[2 col], orand[2 col + 1]).
__global__ void k_cols_orand(Cols in, int ncols, int64_t n, unsigned long long* orand) {
    __shared__ unsigned long long s_or[kMaxCols], s_and[kMaxCols];
    if (threadIdx.x < kMaxCols) {
        s_or[threadIdx.x] = 0ull;
        s_and[threadIdx.x] = ~0ull;
    }
    __syncthreads();
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int k = 0; k < ncols; ++k) {
        unsigned long long o = 0ull, a = ~0ull;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
            const uint64_t v = in.c[k][i];
            o |= v;
            a &= v;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            o |= __shfl_down_sync(0xFFFFFFFFu, o, d);
            a &= __shfl_down_sync(0xFFFFFFFFu, a, d);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicOr(&s_or[k], o);
            atomicAnd(&s_and[k], a);
        }
    }
    __syncthreads();
    if (threadIdx.x < ncols) {
        atomicOr(&orand[2 * threadIdx.x], s_or[threadIdx.x]);
        atomicAnd(&orand[2 * threadIdx.x + 1], s_and[threadIdx.x]);
    }
}

__global__ void k_digit_hist(const uint64_t* __restrict__ key, int shift, int64_t n, uint32_t* hist, int64_t nb) {
    __shared__ uint32_t h[kBins];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kItems; ++r) {
        const int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(key[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of one value per thread over the block (warp_tot: one per warp).
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t* warp_tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < wid; ++w) before += warp_tot[w];
    __syncthreads();
    return before + x - v;
}

// Stable scatter of all columns by one digit of column `kc` (offsets: the
// scanned histogram).  The tile's elements are staged in shared memory in
// digit order (dynamic shared memory: NC columns of kTile words) and written
// out in runs, so that consecutive threads write consecutive addresses.
template <int NC>
__global__ void __launch_bounds__(kThreads) k_digit_scatter(Cols in, Cols out, int kc, int shift, int64_t n,
                                                            const uint32_t* __restrict__ offsets, int64_t nb) {
    extern __shared__ __align__(16) uint64_t st[];  // [NC][kTile]
    __shared__ uint32_t s_wh[kWarps][kBins];
    __shared__ uint32_t s_glob[kBins], s_tile_off[kBins], s_warp[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kTile;
    const int64_t wbase = base + (int64_t)wid * (kItems * 32);
    for (int d = lane; d < kBins; d += 32) s_wh[wid][d] = 0;
    __syncwarp();
    uint32_t pk[kItems];
    const uint64_t* key = nullptr;
#pragma unroll
    for (int k = 0; k < NC; ++k)
        if (k == kc) key = in.c[k];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t i = wbase + (int64_t)r * 32 + lane;
        const uint32_t d = i < n ? ((uint32_t)(key[i] >> shift) & 255u) : (uint32_t)kBins;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (d < kBins && lane == leader) {
            before = s_wh[wid][d];
            s_wh[wid][d] = before + __popc(peers);
        }
        before = __shfl_sync(0xFFFFFFFFu, before, leader);
        __syncwarp();
        pk[r] = (d << 16) | (before + __popc(peers & lt));
    }
    __syncthreads();
    // digit t: offsets of the warps inside the tile's run of t, the run's place in
    // the tile, and its global start
    uint32_t tot = 0;
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = s_wh[w][threadIdx.x];
        s_wh[w][threadIdx.x] = tot;
        tot += c;
    }
    s_tile_off[threadIdx.x] = block_scan(tot, s_warp);
    s_glob[threadIdx.x] = offsets[(int64_t)threadIdx.x * nb + blockIdx.x];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const uint32_t d = pk[r] >> 16;
        if (d >= kBins) continue;
        const int64_t i = wbase + (int64_t)r * 32 + lane;
        const uint32_t pos = s_tile_off[d] + s_wh[wid][d] + (pk[r] & 0xFFFFu);
#pragma unroll
        for (int k = 0; k < NC; ++k) st[k * kTile + pos] = in.c[k][i];
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)kTile, n - base);
    for (int t = threadIdx.x; t < cnt; t += kThreads) {
        const uint32_t d = (uint32_t)(st[kc * kTile + t] >> shift) & 255u;
        const int64_t pos = (int64_t)s_glob[d] + (t - (int64_t)s_tile_off[d]);
#pragma unroll
        for (int k = 0; k < NC; ++k) out.c[k][pos] = st[k * kTile + t];
    }
}

// The sorted columns into the export layout: x [k][W], z [k][W], coef [k].
__global__ void k_cols_to_export(Cols in, int W, int Wd, int64_t k, uint64_t* x, uint64_t* z, double* c) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += s) {
        for (int w = 0; w < W; ++w) {
            x[i * W + w] = in.c[w][i];
            z[i * W + w] = in.c[Wd + w][i];
        }
        c[i] = __longlong_as_double((long long)in.c[2 * Wd][i]);
    }
}

int grid_blocks(int64_t n) {
    int64_t want = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

// Each column takes align_up(8 n) bytes; the two buffers hold ncols columns each.
size_t export_sort_scratch_bytes(int Wd, int64_t n) {
    const int ncols = 2 * Wd + 1;
    const int64_t nb = std::max<int64_t>((n + kTile - 1) / kTile, 1);
    return 2 * (size_t)ncols * align_up((size_t)n * 8) + align_up((size_t)kBins * nb * 4) + 4096 + 1024;
}

// Sort rows [0, n) with their coefficients in canonical order and write the
// first k of them as x [k][W], z [k][W], coef [k] inside scratch
// (export_sort_scratch_bytes(Wd, n)); *out_x, *out_z, *out_c point at them.
void launch_export_sort(int W, int Wd, const uint64_t* rows, const double* coef, int64_t n, int64_t k, void* scratch,
                        uint64_t** out_x, uint64_t** out_z, double** out_c, cudaStream_t s) {
    const int ncols = 2 * Wd + 1;
    const int64_t nb = std::max<int64_t>((n + kTile - 1) / kTile, 1);
    const size_t col = align_up((size_t)n * 8);
    const size_t half = (size_t)ncols * col;
    char* p = (char*)scratch;
    Cols a{}, b{};
    for (int c = 0; c < ncols; ++c) {
        a.c[c] = (uint64_t*)(p + (size_t)c * col);
        b.c[c] = (uint64_t*)(p + half + (size_t)c * col);
    }
    uint32_t* hist = (uint32_t*)(p + 2 * half);
    uint32_t* tmp = (uint32_t*)(p + 2 * half + align_up((size_t)kBins * nb * 4));
    unsigned long long* orand = (unsigned long long*)((char*)tmp + 4096);
    const int g = grid_blocks(n);
    if (n > 0) {
        k_rows_to_cols<<<g, kThreads, 0, s>>>(rows, coef, 2 * Wd, n, a);
        note_launch();
        cudaFuncSetAttribute(k_digit_scatter<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * kTile * 8);
        cudaFuncSetAttribute(k_digit_scatter<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, 5 * kTile * 8);
        cudaFuncSetAttribute(k_digit_scatter<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, 9 * kTile * 8);
        unsigned long long init[2 * kMaxCols];
        for (int c = 0; c < kMaxCols; ++c) {
            init[2 * c] = 0ull;
            init[2 * c + 1] = ~0ull;
        }
        cudaMemcpyAsync(orand, init, sizeof init, cudaMemcpyHostToDevice, s);
        k_cols_orand<<<g, kThreads, 0, s>>>(a, 2 * Wd, n, orand);
        note_launch();
        unsigned long long host[2 * kMaxCols];
        cudaMemcpyAsync(host, orand, sizeof host, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        int order[2 * 4];
        int no = 0;
        for (int w = 0; w < Wd; ++w) order[no++] = Wd + w;  // z words, least significant first
        for (int w = 0; w < Wd; ++w) order[no++] = w;       // then x words
        for (int oi = 0; oi < no; ++oi) {
            const int kc = order[oi];
            const uint64_t varying = host[2 * kc] ^ host[2 * kc + 1];
            for (int shift = 0; shift < 64; shift += 8) {
                if (((varying >> shift) & 255ull) == 0) continue;
                k_digit_hist<<<(unsigned)nb, kThreads, 0, s>>>(a.c[kc], shift, n, hist, nb);
                note_launch();
                launch_scan_u32_long(hist, (int64_t)kBins * nb, tmp, s);
                const size_t smem = (size_t)ncols * kTile * 8;
                if (ncols == 3) k_digit_scatter<3><<<(unsigned)nb, kThreads, smem, s>>>(a, b, kc, shift, n, hist, nb);
                else if (ncols == 5) k_digit_scatter<5><<<(unsigned)nb, kThreads, smem, s>>>(a, b, kc, shift, n, hist, nb);
                else k_digit_scatter<9><<<(unsigned)nb, kThreads, smem, s>>>(a, b, kc, shift, n, hist, nb);
                note_launch();
                const Cols t = a;
                a = b;
                b = t;
            }
        }
    }
    // the export layout into the other buffer
    uint64_t* x = b.c[0];
    uint64_t* z = x + (size_t)k * W;
    double* c = (double*)(z + (size_t)k * W);
    if (k > 0) {
        k_cols_to_export<<<grid_blocks(k), kThreads, 0, s>>>(a, W, Wd, k, x, z, c);
        note_launch();
    }
    *out_x = x;
    *out_z = z;
    *out_c = c;
}

}  // namespace iqcc
