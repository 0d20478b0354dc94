// Direct stable LSD radix sort of the rows in canonical order, for export.
//
// The rows are split into columns (x words, z words, the coefficient's bits)
// and every pass moves whole columns: per tile of 1024 elements a histogram of
// one 8-bit digit, a multi-block exclusive scan over (digit, tile), and a
// stable scatter whose ranks come from warp-local counters (each warp owns 128
// consecutive elements; lanes with the same digit find each other with
// match_any) and whose writes are staged in shared memory in digit order, so
// no key is ever gathered through a permutation and writes leave in runs.
// Digits that are constant over all elements are skipped.  Canonical order
// compares x as an integer with its last word most significant, then z
// likewise, so the passes run over z_0, ..., z_{Wd-1}, then x_0, ..., x_{Wd-1},
// low byte first.
//
// Rows keep their relative order through dressing and compaction, so a table
// that was loaded in canonical order is still sorted up to its first appended
// term.  The longest sorted prefix is found first; only the rest is radix
// sorted, and the two sorted runs are merged tile by tile straight into the
// export layout (merge path: the split of every tile boundary by binary
// search, then inside a tile every element's place is its index in its own run
// plus its rank in the other run).  The merge writes page-locked host memory
// directly when given it; into device scratch it needs the prefix to hold
// about half of the rows (else all rows are sorted).
#include <cuda_runtime.h>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 4;
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
// Sorted columns into the export layout.  Consecutive threads write
// consecutive words (the destination may be pinned host memory).
__global__ void k_cols_to_export(Cols in, int W, int Wd, int64_t k, uint64_t* x, uint64_t* z, double* c) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    const int64_t kw = k * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < kw; i += s) {
        const int64_t o = i / W;
        const int w = (int)(i - o * W);
        x[i] = in.c[w][o];
        z[i] = in.c[Wd + w][o];
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += s)
        c[i] = __longlong_as_double((long long)in.c[2 * Wd][i]);
}

// Smallest i in [1, n) whose row is not above row i - 1 in canonical order
// (atomic minimum into *first, which starts at n): rows [0, i) are sorted.
template <int WD>
__global__ void k_first_descent(const uint64_t* __restrict__ rows, int64_t n, unsigned long long* first) {
    unsigned long long best = (unsigned long long)n;
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        const Key<WD> a = load_key<WD>(rows, i - 1), b = load_key<WD>(rows, i);
        int cmp = 0;
#pragma unroll
        for (int w = WD - 1; w >= 0; --w)
            if (!cmp && a.x[w] != b.x[w]) cmp = a.x[w] < b.x[w] ? -1 : 1;
#pragma unroll
        for (int w = WD - 1; w >= 0; --w)
            if (!cmp && a.z[w] != b.z[w]) cmp = a.z[w] < b.z[w] ? -1 : 1;
        if (cmp >= 0) {
            best = (unsigned long long)i;
            break;  // a thread's indices rise, so its first hit is its smallest
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(0xFFFFFFFFu, best, o));
    if ((threadIdx.x & 31) == 0 && best < (unsigned long long)n) atomicMin(first, best);
}

constexpr int kMergeTile = 1024;

// Row i of the sorted prefix (rows, 2 WD words) below element j of the sorted columns.
template <int WD>
__device__ __forceinline__ bool row_below_col(const uint64_t* __restrict__ rows, int64_t i, const Cols& a, int64_t j) {
    const uint64_t* r = rows + (size_t)i * 2 * WD;
#pragma unroll
    for (int w = WD - 1; w >= 0; --w) {
        const uint64_t p = r[w], q = a.c[w][j];
        if (p != q) return p < q;
    }
#pragma unroll
    for (int w = WD - 1; w >= 0; --w) {
        const uint64_t p = r[WD + w], q = a.c[WD + w][j];
        if (p != q) return p < q;
    }
    return false;
}

// Merge path: split[t] = number of prefix rows among the first min(t T, k)
// outputs of the merge of the prefix [0, P) with the sorted columns [0, m).
template <int WD>
__global__ void k_merge_splits(const uint64_t* __restrict__ rows, int64_t P, Cols a, int64_t m, int64_t k, int64_t nt,
                               int64_t* split) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= nt; t += s) {
        const int64_t d = min(t * kMergeTile, k);
        int64_t lo = max((int64_t)0, d - m), hi = min(d, P);
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (row_below_col<WD>(rows, mid, a, d - 1 - mid)) lo = mid + 1;
            else hi = mid;
        }
        split[t] = lo;
    }
}

// Shared-memory element e below element f (columns of kMergeTile words).
template <int WD>
__device__ __forceinline__ bool tile_below(const uint64_t* sk, int e, int f) {
#pragma unroll
    for (int w = WD - 1; w >= 0; --w) {
        const uint64_t p = sk[w * kMergeTile + e], q = sk[w * kMergeTile + f];
        if (p != q) return p < q;
    }
#pragma unroll
    for (int w = WD - 1; w >= 0; --w) {
        const uint64_t p = sk[(WD + w) * kMergeTile + e], q = sk[(WD + w) * kMergeTile + f];
        if (p != q) return p < q;
    }
    return false;
}

// One output tile of the merge, written in the export layout.  The tile's
// prefix rows occupy shared-memory elements [0, np), its sorted-column elements
// [np, cnt); keys are distinct, so the places form a permutation of the tile.
template <int WD>
__global__ void __launch_bounds__(kThreads) k_merge_export(const uint64_t* __restrict__ rows,
                                                           const double* __restrict__ coef, Cols a,
                                                           const int64_t* __restrict__ split, int64_t k, int W,
                                                           uint64_t* x, uint64_t* z, double* c) {
    constexpr int S = 2 * WD;
    extern __shared__ __align__(16) uint64_t sk[];  // [S + 1][kMergeTile]
    __shared__ uint16_t place[kMergeTile];
    const int64_t d0 = (int64_t)blockIdx.x * kMergeTile;
    const int cnt = (int)min((int64_t)kMergeTile, k - d0);
    const int64_t i0 = split[blockIdx.x];
    const int np = (int)(split[blockIdx.x + 1] - i0);
    const int na = cnt - np;
    const int64_t j0 = d0 - i0;
    for (int f = threadIdx.x; f < np * S; f += kThreads) sk[(f % S) * kMergeTile + f / S] = rows[i0 * S + f];
    for (int e = threadIdx.x; e < np; e += kThreads)
        sk[S * kMergeTile + e] = (uint64_t)__double_as_longlong(coef[i0 + e]);
    for (int e = threadIdx.x; e < na; e += kThreads) {
#pragma unroll
        for (int col = 0; col <= S; ++col) sk[col * kMergeTile + np + e] = a.c[col][j0 + e];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += kThreads) {
        const bool pre = e < np;
        const int base = pre ? np : 0;
        int lo = 0, hi = pre ? na : np;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (tile_below<WD>(sk, base + mid, e)) lo = mid + 1;
            else hi = mid;
        }
        place[(pre ? e : e - np) + lo] = (uint16_t)e;
    }
    __syncthreads();
    // consecutive threads write consecutive words (the destination may be pinned host memory)
    for (int f = threadIdx.x; f < cnt * W; f += kThreads) {
        const int t = f / W, w = f - t * W;
        const int e = place[t];
        x[d0 * W + f] = sk[w * kMergeTile + e];
        z[d0 * W + f] = sk[(WD + w) * kMergeTile + e];
    }
    for (int t = threadIdx.x; t < cnt; t += kThreads)
        c[d0 + t] = __longlong_as_double((long long)sk[S * kMergeTile + place[t]]);
}

// The first k rows (already in canonical order) in the export layout.
__global__ void k_rows_to_export(const uint64_t* __restrict__ rows, const double* __restrict__ coef, int W, int Wd,
                                 int64_t k, uint64_t* x, uint64_t* z, double* c) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    const int64_t kw = k * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < kw; i += s) {
        const int64_t o = i / W;
        const int w = (int)(i - o * W);
        x[i] = rows[o * 2 * Wd + w];
        z[i] = rows[o * 2 * Wd + Wd + w];
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += s) c[i] = coef[i];
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

namespace {

// Stable LSD radix sort of rows [0, n) with their coefficients into canonical
// order, through the column buffers a and b; returns the one holding the result.
Cols radix_sort_cols(int Wd, const uint64_t* rows, const double* coef, int64_t n, Cols a, Cols b, uint32_t* hist,
                     uint32_t* tmp, unsigned long long* orand, cudaStream_t s) {
    const int ncols = 2 * Wd + 1;
    const int64_t nb = std::max<int64_t>((n + kTile - 1) / kTile, 1);
    const int g = grid_blocks(n);
    k_rows_to_cols<<<g, kThreads, 0, s>>>(rows, coef, 2 * Wd, n, a);
    note_launch();
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
    const size_t smem = (size_t)ncols * kTile * 8;
    for (int oi = 0; oi < no; ++oi) {
        const int kc = order[oi];
        const uint64_t varying = host[2 * kc] ^ host[2 * kc + 1];
        for (int shift = 0; shift < 64; shift += 8) {
            if (((varying >> shift) & 255ull) == 0) continue;
            k_digit_hist<<<(unsigned)nb, kThreads, 0, s>>>(a.c[kc], shift, n, hist, nb);
            note_launch();
            launch_scan_u32_long(hist, (int64_t)kBins * nb, tmp, s);
            if (ncols == 3) k_digit_scatter<3><<<(unsigned)nb, kThreads, smem, s>>>(a, b, kc, shift, n, hist, nb);
            else if (ncols == 5) k_digit_scatter<5><<<(unsigned)nb, kThreads, smem, s>>>(a, b, kc, shift, n, hist, nb);
            else k_digit_scatter<9><<<(unsigned)nb, kThreads, smem, s>>>(a, b, kc, shift, n, hist, nb);
            note_launch();
            const Cols t = a;
            a = b;
            b = t;
        }
    }
    return a;
}

void set_smem_limits() {
    static std::atomic<unsigned long long> done{0};
    if (!first_on_device(&done)) return;
    cudaFuncSetAttribute(k_digit_scatter<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * kTile * 8);
    cudaFuncSetAttribute(k_digit_scatter<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, 5 * kTile * 8);
    cudaFuncSetAttribute(k_digit_scatter<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, 9 * kTile * 8);
    cudaFuncSetAttribute(k_merge_export<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * kMergeTile * 8);
    cudaFuncSetAttribute(k_merge_export<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 5 * kMergeTile * 8);
    cudaFuncSetAttribute(k_merge_export<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 9 * kMergeTile * 8);
}

}  // namespace

// Sort rows [0, n) with their coefficients in canonical order and write the
// first k of them as x [k][W], z [k][W], coef [k].  With dst_x, dst_z, dst_c
// all non-null (addresses the device can write: device memory or mapped
// pinned host memory) the layout goes there; otherwise it is placed inside
// scratch.  *out_x, *out_z, *out_c receive where it was written.
//
// Scratch (export_sort_scratch_bytes(Wd, n)): two halves of ncols columns of
// align_up(8 n) bytes, then the histogram, the scan's partials and the OR/AND
// words.  The sorted prefix [0, P) is found first.  When the rest [P, n) can be
// sorted in two column sets of align_up(8 (n - P)) bytes while the layout has
// its own room (a direct destination, or the first half when n - P is at most
// about n / 2), only the rest is sorted and merged with the prefix; otherwise
// all rows are sorted, ping-ponging between the halves, and the layout goes
// into the half the sort does not end in.
void launch_export_sort(int W, int Wd, const uint64_t* rows, const double* coef, int64_t n, int64_t k, void* scratch,
                        uint64_t* dst_x, uint64_t* dst_z, double* dst_c, uint64_t** out_x, uint64_t** out_z,
                        double** out_c, cudaStream_t s) {
    const int ncols = 2 * Wd + 1;
    const int64_t nb = std::max<int64_t>((n + kTile - 1) / kTile, 1);
    const size_t col = align_up((size_t)n * 8);
    const size_t half = (size_t)ncols * col;
    char* p = (char*)scratch;
    uint32_t* hist = (uint32_t*)(p + 2 * half);
    uint32_t* tmp = (uint32_t*)(p + 2 * half + align_up((size_t)kBins * nb * 4));
    unsigned long long* orand = (unsigned long long*)((char*)tmp + 4096);
    set_smem_limits();
    const bool direct = dst_x && dst_z && dst_c;
    // the sorted prefix
    int64_t P = n;
    if (n > 1) {
        const unsigned long long init = (unsigned long long)n;
        cudaMemcpyAsync(orand, &init, 8, cudaMemcpyHostToDevice, s);
        const int g = grid_blocks(n);
        if (Wd == 1) k_first_descent<1><<<g, kThreads, 0, s>>>(rows, n, orand);
        else if (Wd == 2) k_first_descent<2><<<g, kThreads, 0, s>>>(rows, n, orand);
        else k_first_descent<4><<<g, kThreads, 0, s>>>(rows, n, orand);
        note_launch();
        unsigned long long first = 0;
        cudaMemcpyAsync(&first, orand, 8, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        P = (int64_t)first;
    }
    const int64_t m = n - P;
    const size_t colm = align_up((size_t)m * 8);
    uint64_t* x = direct ? dst_x : (uint64_t*)p;  // the first half unless the full sort ends there
    uint64_t* z = direct ? dst_z : x + (size_t)k * W;
    double* c = direct ? dst_c : (double*)(x + 2 * (size_t)k * W);
    if (m == 0) {
        if (k > 0) {
            k_rows_to_export<<<grid_blocks(k * W), kThreads, 0, s>>>(rows, coef, W, Wd, k, x, z, c);
            note_launch();
        }
    } else if (direct || 2 * colm <= col) {
        // rest sorted in the second half (a direct destination leaves both halves to it)
        char* base = direct ? p : p + half;
        Cols a{}, b{};
        for (int j = 0; j < ncols; ++j) {
            a.c[j] = (uint64_t*)(base + (size_t)j * colm);
            b.c[j] = (uint64_t*)(base + (size_t)(ncols + j) * colm);
        }
        const Cols sorted = radix_sort_cols(Wd, rows + (size_t)P * 2 * Wd, coef + P, m, a, b, hist, tmp, orand, s);
        if (k > 0) {
            const int64_t nt = (k + kMergeTile - 1) / kMergeTile;
            int64_t* split = (int64_t*)hist;  // the histogram is free once the sort is done
            const int gs = grid_blocks(nt + 1);
            const size_t smem = (size_t)ncols * kMergeTile * 8;
            if (Wd == 1) {
                k_merge_splits<1><<<gs, kThreads, 0, s>>>(rows, P, sorted, m, k, nt, split);
                k_merge_export<1><<<(unsigned)nt, kThreads, smem, s>>>(rows, coef, sorted, split, k, W, x, z, c);
            } else if (Wd == 2) {
                k_merge_splits<2><<<gs, kThreads, 0, s>>>(rows, P, sorted, m, k, nt, split);
                k_merge_export<2><<<(unsigned)nt, kThreads, smem, s>>>(rows, coef, sorted, split, k, W, x, z, c);
            } else {
                k_merge_splits<4><<<gs, kThreads, 0, s>>>(rows, P, sorted, m, k, nt, split);
                k_merge_export<4><<<(unsigned)nt, kThreads, smem, s>>>(rows, coef, sorted, split, k, W, x, z, c);
            }
            note_launch();
            note_launch();
        }
    } else {
        Cols a{}, b{};
        for (int j = 0; j < ncols; ++j) {
            a.c[j] = (uint64_t*)(p + (size_t)j * col);
            b.c[j] = (uint64_t*)(p + half + (size_t)j * col);
        }
        const Cols sorted = radix_sort_cols(Wd, rows, coef, n, a, b, hist, tmp, orand, s);
        if (!direct) {
            x = sorted.c[0] == a.c[0] ? b.c[0] : a.c[0];
            z = x + (size_t)k * W;
            c = (double*)(x + 2 * (size_t)k * W);
        }
        if (k > 0) {
            k_cols_to_export<<<grid_blocks(k * W), kThreads, 0, s>>>(sorted, W, Wd, k, x, z, c);
            note_launch();
        }
    }
    *out_x = x;
    *out_z = z;
    *out_c = c;
}

}  // namespace iqcc
