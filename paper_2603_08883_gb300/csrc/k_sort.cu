// Reordering kernels: indirect stable LSD radix sort on multi-word keys,
// stable stream compaction, load-time canonicalisation (sort + segmented sum
// of repeated keys, Eq. 2), export in canonical order, compression flags
// (magnitude threshold and term budget by radix select on the |C| bit
// pattern), and the DIS candidate ordering.
#include <cuda_runtime.h>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // elements per block in sort / compaction

int64_t n_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

// ---------------------------------------------------------------- radix sort

__global__ void k_word_orand(const uint64_t* __restrict__ keys, int stride, const uint32_t* __restrict__ perm,
                             int64_t n, unsigned long long* orand /* [2*stride] */) {
    // per-word OR and AND over the listed elements (to skip constant digits)
    extern __shared__ unsigned long long sh[];
    for (int w = threadIdx.x; w < 2 * stride; w += blockDim.x) sh[w] = (w < stride) ? 0ull : ~0ull;
    __syncthreads();
    unsigned long long o[9], a[9];
    for (int w = 0; w < stride; ++w) { o[w] = 0ull; a[w] = ~0ull; }
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        const uint64_t* k = keys + (size_t)perm[i] * stride;
        for (int w = 0; w < stride; ++w) { o[w] |= k[w]; a[w] &= k[w]; }
    }
    for (int w = 0; w < stride; ++w) {
        atomicOr(sh + w, o[w]);
        atomicAnd(sh + stride + w, a[w]);
    }
    __syncthreads();
    for (int w = threadIdx.x; w < 2 * stride; w += blockDim.x) {
        if (w < stride) atomicOr(orand + w, sh[w]);
        else atomicAnd(orand + w, sh[w]);
    }
}

__global__ void k_sort_hist(const uint64_t* __restrict__ keys, int stride, int word, int shift,
                            const uint32_t* __restrict__ perm, int64_t n, uint32_t* hist, int64_t nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kItems; ++r) {
        int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
        if (i < n) {
            uint32_t d = (uint32_t)(keys[(size_t)perm[i] * stride + word] >> shift) & 255u;
            atomicAdd(&h[d], 1u);
        }
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of a u32 array in place by one block (n up to a few million).
__global__ void k_scan_u32(uint32_t* data, int64_t n) {
    __shared__ uint32_t sums[1024];
    const int T = blockDim.x;
    const int64_t chunk = (n + T - 1) / T;
    const int64_t lo = threadIdx.x * chunk, hi = min(n, lo + chunk);
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += data[i];
    sums[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        uint32_t v = threadIdx.x >= off ? sums[threadIdx.x - off] : 0u;
        __syncthreads();
        sums[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? sums[threadIdx.x - 1] : 0u;
    for (int64_t i = lo; i < hi; ++i) {
        uint32_t v = data[i];
        data[i] = run;
        run += v;
    }
}

// Stable scatter of one digit: rounds of 256 elements in index order; within a
// round warps in order and lanes in order (match_any gives the same-digit peers).
__global__ void k_sort_scatter(const uint64_t* __restrict__ keys, int stride, int word, int shift,
                               const uint32_t* __restrict__ perm_in, uint32_t* perm_out, int64_t n,
                               const uint32_t* __restrict__ offsets, int64_t nblocks) {
    __shared__ uint32_t s_off[256];
    __shared__ uint32_t s_cnt[kThreads / 32][256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    s_off[threadIdx.x] = offsets[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kItems; ++r) {
        for (int w = 0; w < kThreads / 32; ++w) s_cnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
        const bool valid = i < n;
        uint32_t src = 0, d = 256;
        if (valid) {
            src = perm_in[i];
            d = (uint32_t)(keys[(size_t)src * stride + word] >> shift) & 255u;
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) s_cnt[wid][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = s_off[d] + rank;
            for (int w = 0; w < wid; ++w) pos += s_cnt[w][d];
            perm_out[pos] = src;
        }
        __syncthreads();
        uint32_t tot = 0;
        for (int w = 0; w < kThreads / 32; ++w) tot += s_cnt[w][threadIdx.x];
        s_off[threadIdx.x] += tot;
        __syncthreads();
    }
}

__global__ void k_iota(uint32_t* p, int64_t n) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) p[i] = (uint32_t)i;
}

// ---------------------------------------------------------------- compaction

__global__ void k_flag_count(const uint8_t* __restrict__ flags, int64_t n, uint32_t* counts) {
    __shared__ uint32_t s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    uint32_t c = 0;
    for (int r = 0; r < kItems; ++r) {
        int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
        if (i < n && flags[i]) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = s;
}

__global__ void k_total(const uint32_t* scanned, const uint32_t* counts_last, int64_t nb,
                        unsigned long long* total) {
    *total = (unsigned long long)scanned[nb - 1] + (unsigned long long)*counts_last;
}

template <int W>
__global__ void k_compact_scatter(const uint8_t* __restrict__ flags, const uint64_t* __restrict__ rows_in,
                                  const double* __restrict__ c_in, uint64_t* rows_out, double* c_out, int64_t n,
                                  const uint32_t* __restrict__ offsets) {
    __shared__ uint32_t s_w[kThreads / 32];
    __shared__ uint32_t s_base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_base = offsets[blockIdx.x];
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kItems; ++r) {
        const int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
        const bool f = i < n && flags[i];
        const unsigned b = __ballot_sync(0xFFFFFFFFu, f);
        if (lane == 0) s_w[wid] = __popc(b);
        __syncthreads();
        uint32_t pos = s_base + __popc(b & ((1u << lane) - 1u));
        for (int w = 0; w < wid; ++w) pos += s_w[w];
        if (f) {
            Key<W> k = load_key<W>(rows_in, i);
            store_key<W>(rows_out, pos, k);
            c_out[pos] = c_in[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < kThreads / 32; ++w) t += s_w[w];
            s_base += t;
        }
        __syncthreads();
    }
}

// Single-pass stable in-place compaction (decoupled look-back).  Tiles take
// ids in launch order from a counter.  Each warp of a tile reads its own 128
// consecutive rows (the keys and coefficients of kept rows only) into
// registers and ranks them with ballots; the tile publishes its count, sums
// its predecessors' counts 32 at a time with its first warp (waiting, with a
// bound, for any not yet published), publishes its inclusive prefix and only
// then writes, straight from registers.  Its destination [prefix, prefix + count) lies below the
// end of its own rows, its own rows were all read before the barrier that
// precedes the writes, and every earlier tile read its rows before
// publishing, so no row is overwritten before it is read.
constexpr int kCompactTile = 1024;  // rows per tile (4 per thread)
constexpr unsigned long long kStAgg = 1ull << 62, kStPrefix = 2ull << 62;
constexpr unsigned long long kStMask = (1ull << 62) - 1;

template <int W>
__global__ void __launch_bounds__(kThreads) k_compact_inplace(const uint8_t* __restrict__ flags, uint64_t* rows,
                                                              double* coef, int64_t n,
                                                              unsigned long long* state,
                                                              unsigned int* tile_counter,
                                                              unsigned long long* total, DevCounters* ctr,
                                                              uint32_t* new_row) {
    constexpr int kPer = kCompactTile / kThreads;
    __shared__ uint32_t s_w[kThreads / 32];  // warp counts, then warp offsets within the tile
    __shared__ unsigned int s_tile;
    __shared__ unsigned long long s_prefix;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const unsigned int t = s_tile;
    const int64_t base = (int64_t)t * kCompactTile;
    const int64_t wbase = base + (int64_t)wid * (kPer * 32);
    Key<W> key[kPer];
    double c[kPer];
    uint32_t rank[kPer];
    bool keep[kPer];
    uint32_t wcount = 0;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int64_t i = wbase + (int64_t)r * 32 + lane;
        keep[r] = i < n && flags[i];
        if (keep[r]) {
            key[r] = load_key<W>(rows, i);
            c[r] = coef[i];
        }
        const unsigned b = __ballot_sync(0xFFFFFFFFu, keep[r]);
        rank[r] = wcount + __popc(b & lt);
        wcount += __popc(b);
    }
    if (lane == 0) s_w[wid] = wcount;
    __syncthreads();
    if (wid == 0) {
        // warp offsets within the tile and the tile's count
        const uint32_t v = lane < kThreads / 32 ? s_w[lane] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t count = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (lane < kThreads / 32) s_w[lane] = incl - v;
        if (lane == 0) {
            __threadfence();
            atomicExch(state + t, (t == 0 ? kStPrefix : kStAgg) | count);
        }
        // look back 32 predecessors at a time: sum their aggregates up to the
        // closest one that has published its inclusive prefix
        unsigned long long prefix = 0;
        int64_t p = (int64_t)t - 1;
        int spins = 0;
        while (p >= 0) {
            const int64_t q = p - lane;
            unsigned long long v2 = kStPrefix | 0ull;  // before tile 0: a prefix of 0
            if (q >= 0) v2 = *(volatile unsigned long long*)(state + q);
            const unsigned pref = __ballot_sync(0xFFFFFFFFu, (v2 & ~kStMask) == kStPrefix);
            const unsigned zero = __ballot_sync(0xFFFFFFFFu, v2 == 0);
            const int stop = pref ? __ffs(pref) - 1 : 31;  // last lane that counts
            const unsigned upto = stop == 31 ? 0xFFFFFFFFu : ((2u << stop) - 1u);
            if (zero & upto) {  // a predecessor within the window has not published yet
                if (++spins > ctr->wait_limit) {
                    if (lane == 0 && atomicCAS(&ctr->err, 0, (int)IQCC_ERR_TIMEOUT) == 0) ctr->err_where = 20;
                    break;
                }
                __nanosleep(32);
                continue;
            }
            unsigned long long part = lane <= stop ? (v2 & kStMask) : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xFFFFFFFFu, part, o);
            prefix += __shfl_sync(0xFFFFFFFFu, part, 0);
            if (pref) break;
            p -= 32;
        }
        if (lane == 0) {
            if (t != 0) atomicExch(state + t, kStPrefix | (prefix + count));
            s_prefix = prefix;
            if (base + kCompactTile >= n) *total = prefix + count;  // last tile
        }
    }
    __syncthreads();
    const unsigned long long out = s_prefix + s_w[wid];
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int64_t i = wbase + (int64_t)r * 32 + lane;
        if (keep[r]) {
            store_key<W>(rows, (int64_t)(out + rank[r]), key[r]);
            coef[out + rank[r]] = c[r];
        }
        if (new_row && i < n) new_row[i] = keep[r] ? (uint32_t)(out + rank[r]) : kRowRemoved;
    }
}

// One bounded device wait on a word that nothing writes: polls until the
// context's wait limit is spent, then records IQCC_ERR_TIMEOUT and returns
// (the failure path every device wait of the library takes).
__global__ void k_wait_selftest(const unsigned long long* word, DevCounters* ctr) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int spins = 0;
    while (*(const volatile unsigned long long*)word == 0) {
        if (++spins > ctr->wait_limit) {
            set_error(ctr, IQCC_ERR_TIMEOUT, 90);
            return;
        }
        __nanosleep(32);
    }
}

// Coarse |g| (20 low mantissa bits cleared) digit histogram of all groups.
__global__ void k_coarse_digit_hist(const double* __restrict__ g, int64_t G, int shift, uint64_t prefix,
                                    uint64_t prefix_mask, unsigned long long* hist) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < G; i += s) {
        const uint64_t b = ((uint64_t)__double_as_longlong(g[i]) & 0x7FFFFFFFFFFFFFFFull) & ~((1ull << 20) - 1ull);
        if ((b & prefix_mask) != prefix) continue;
        atomicAdd(&h[(b >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(hist + threadIdx.x, (unsigned long long)h[threadIdx.x]);
}

// Indices of groups whose coarse |g| >= t (at most cap of them are written).
__global__ void k_collect_ge(const double* __restrict__ g, int64_t G, uint64_t t, uint32_t* idx, int64_t cap,
                             unsigned long long* count) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < G; i += s) {
        const uint64_t b = ((uint64_t)__double_as_longlong(g[i]) & 0x7FFFFFFFFFFFFFFFull) & ~((1ull << 20) - 1ull);
        if (b < t) continue;
        const unsigned long long k = atomicAdd(count, 1ull);
        if ((int64_t)k < cap) idx[k] = (uint32_t)i;
    }
}

// skeys for a listed subset of groups (same layout as k_dis_sort_keys).
__global__ void k_dis_sort_keys_sub(int Wd, const uint64_t* __restrict__ gkeys, const double* __restrict__ gsum,
                                    const uint32_t* __restrict__ idx, int64_t k, uint64_t* skeys) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += s) {
        const uint32_t g = idx[i];
        uint64_t a = ((uint64_t)__double_as_longlong(gsum[g]) & 0x7FFFFFFFFFFFFFFFull) & ~((1ull << 20) - 1ull);
        skeys[(size_t)i * (Wd + 1)] = ~a;  // compact: entry i is the i-th listed group
        for (int w = 0; w < Wd; ++w) skeys[(size_t)i * (Wd + 1) + 1 + w] = gkeys[(size_t)g * Wd + (Wd - 1 - w)];
    }
}

// ---------------------------------------------------------------- load / export

// Host layout (x [n][W], z [n][W]) to device rows; keys with bits set in
// hi_mask of their last word (above n_qubits) are counted in *bad.
__global__ void k_pack_rows(int W, int Wd, const uint64_t* __restrict__ x, const uint64_t* __restrict__ z,
                            uint64_t* rows, int64_t n, uint64_t hi_mask, unsigned long long* bad) {
    unsigned long long nbad = 0;
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        for (int w = 0; w < Wd; ++w) {
            rows[(size_t)i * 2 * Wd + w] = w < W ? x[(size_t)i * W + w] : 0ull;
            rows[(size_t)i * 2 * Wd + Wd + w] = w < W ? z[(size_t)i * W + w] : 0ull;
        }
        nbad += ((x[(size_t)i * W + W - 1] | z[(size_t)i * W + W - 1]) & hi_mask) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nbad += __shfl_down_sync(0xFFFFFFFFu, nbad, o);
    if (bad && (threadIdx.x & 31) == 0 && nbad) atomicAdd(bad, nbad);
}

__global__ void k_unpack_rows(int W, int Wd, const uint64_t* __restrict__ rows, const double* __restrict__ coef,
                              const uint32_t* __restrict__ perm, uint64_t* x, uint64_t* z, double* c, int64_t n) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        const uint32_t r = perm ? perm[i] : (uint32_t)i;
        for (int w = 0; w < W; ++w) {
            x[(size_t)i * W + w] = rows[(size_t)r * 2 * Wd + w];
            z[(size_t)i * W + w] = rows[(size_t)r * 2 * Wd + Wd + w];
        }
        c[i] = coef[r];
    }
}

template <int W>
__device__ __forceinline__ bool same_key_rows(const uint64_t* rows, uint32_t a, uint32_t b) {
    Key<W> ka = load_key<W>(rows, a), kb = load_key<W>(rows, b);
    return key_equal<W>(ka, kb);
}

// After the sort: position i starts a run when its key differs from position
// i-1.  The run head sums the run in sorted (= stable input) order and writes
// the key and sum to position i of the gathered output; flags[i] = sum != 0.
template <int W>
__global__ void k_sum_runs(const uint64_t* __restrict__ rows, const double* __restrict__ coef,
                           const uint32_t* __restrict__ perm, int64_t n, uint8_t* flags, uint64_t* rows_out,
                           double* c_out, bool keep_zeros) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        const uint32_t r = perm[i];
        const bool head = (i == 0) || !same_key_rows<W>(rows, perm[i - 1], r);
        if (!head) { flags[i] = 0; continue; }
        double sum = coef[r];
        for (int64_t j = i + 1; j < n && same_key_rows<W>(rows, perm[j], r); ++j) sum += coef[perm[j]];
        Key<W> k = load_key<W>(rows, r);
        store_key<W>(rows_out, i, k);
        c_out[i] = sum;
        flags[i] = keep_zeros || sum != 0.0;
    }
}

// Pairs of consecutive rows not in strictly increasing canonical order (x as
// an integer, last word most significant, then z): zero means the rows are
// sorted and their keys distinct.
template <int W>
__global__ void k_order_violations(const uint64_t* __restrict__ rows, int64_t n, unsigned long long* count) {
    unsigned long long bad = 0;
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        const Key<W> a = load_key<W>(rows, i - 1), b = load_key<W>(rows, i);
        int cmp = 0;
#pragma unroll
        for (int w = W - 1; w >= 0; --w)
            if (!cmp && a.x[w] != b.x[w]) cmp = a.x[w] < b.x[w] ? -1 : 1;
#pragma unroll
        for (int w = W - 1; w >= 0; --w)
            if (!cmp && a.z[w] != b.z[w]) cmp = a.z[w] < b.z[w] ? -1 : 1;
        bad += cmp < 0 ? 0 : 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_down_sync(0xFFFFFFFFu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(count, bad);
}

template <int W>
__global__ void k_gather_rows(const uint64_t* __restrict__ rows, const double* __restrict__ coef,
                              const uint32_t* __restrict__ perm, int64_t n, uint64_t* rows_out, double* c_out) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        const uint32_t r = perm[i];
        store_key<W>(rows_out, i, load_key<W>(rows, r));
        c_out[i] = coef[r];
    }
}

// ---------------------------------------------------------------- compression

__device__ __forceinline__ uint64_t abs_bits(double c) {
    return (uint64_t)__double_as_longlong(c) & 0x7FFFFFFFFFFFFFFFull;
}

__global__ void k_prune_flags(const double* __restrict__ coef, int64_t n, double eps, uint8_t* flags,
                              unsigned long long* count) {
    unsigned c = 0;
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        const bool keep = !(fabs(coef[i]) < eps);
        flags[i] = keep;
        c += keep;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

__global__ void k_abs_digit_hist(const double* __restrict__ coef, const uint8_t* __restrict__ flags, int64_t n,
                                 int shift, uint64_t prefix, uint64_t prefix_mask, unsigned long long* hist) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        if (!flags[i]) continue;
        const uint64_t b = abs_bits(coef[i]);
        if ((b & prefix_mask) != prefix) continue;
        atomicAdd(&h[(b >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(hist + threadIdx.x, (unsigned long long)h[threadIdx.x]);
}

__global__ void k_budget_flags(const double* __restrict__ coef, uint8_t* flags, int64_t n, uint64_t t,
                               uint32_t* tie_idx, unsigned long long* tie_count) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        if (!flags[i]) continue;
        const uint64_t b = abs_bits(coef[i]);
        if (b > t) continue;
        flags[i] = 0;
        if (b == t) tie_idx[atomicAdd(tie_count, 1ull)] = (uint32_t)i;
    }
}

__global__ void k_set_flags(const uint32_t* __restrict__ idx, int64_t k, uint8_t* flags) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += s) flags[idx[i]] = 1;
}

// 12-bit digit histogram of |C| bit patterns among kept rows (every row when
// flags is NULL) whose higher bits equal `prefix` (bits under `prefix_mask`).
__global__ void k_abs_digit_hist12(const double* __restrict__ coef, const uint8_t* __restrict__ flags, int64_t n,
                                   int shift, uint64_t prefix, uint64_t prefix_mask, unsigned long long* hist) {
    __shared__ unsigned int h[4096];
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        if (flags && !flags[i]) continue;
        const uint64_t b = abs_bits(coef[i]);
        if ((b & prefix_mask) != prefix) continue;
        atomicAdd(&h[(b >> shift) & 4095u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4096; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

// The first two levels of the select in one pass when the first level's digit
// is guessed: hist1 over the digit at shift1 of every kept row, hist2 over the
// digit at shift2 of the kept rows whose first digit is `guess`.
__global__ void k_abs_digit_hist12x2(const double* __restrict__ coef, const uint8_t* __restrict__ flags,
                                     int64_t n, int shift1, int shift2, unsigned guess, unsigned long long* hist1,
                                     unsigned long long* hist2) {
    __shared__ unsigned int h1[4096], h2[4096];
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) h1[i] = h2[i] = 0;
    __syncthreads();
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        if (flags && !flags[i]) continue;
        const uint64_t b = abs_bits(coef[i]);
        const unsigned d1 = (unsigned)(b >> shift1) & 4095u;
        atomicAdd(&h1[d1], 1u);
        if (d1 == guess) atomicAdd(&h2[(b >> shift2) & 4095u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) {
        if (h1[i]) atomicAdd(hist1 + i, (unsigned long long)h1[i]);
        if (h2[i]) atomicAdd(hist2 + i, (unsigned long long)h2[i]);
    }
}

// |C| of the kept rows inside the bucket (bits under prefix_mask equal prefix),
// appended to vals (at most cap of them; *n_vals counts them all).
__global__ void k_bucket_values(const double* __restrict__ coef, const uint8_t* __restrict__ flags, int64_t n,
                                uint64_t prefix, uint64_t prefix_mask, double* vals, unsigned long long* n_vals,
                                unsigned long long cap) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        if (!flags[i]) continue;
        const uint64_t b = abs_bits(coef[i]);
        if ((b & prefix_mask) != prefix) continue;
        const unsigned long long k = atomicAdd(n_vals, 1ull);
        if (k < cap) vals[k] = __longlong_as_double((long long)b);
    }
}

// rank[i] = boost for kept rows with |C| >= t (t given by its bit pattern).
__global__ void k_boost_rank(const double* __restrict__ coef, const uint8_t* __restrict__ flags, int64_t n,
                             uint64_t t_bits, double boost, double* rank) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s)
        if (flags[i] && abs_bits(coef[i]) >= t_bits) rank[i] = boost;
}

// Kept rows above the threshold bucket stay kept; rows in it become candidates
// (listed, flag cleared); rows below are dropped.
__global__ void k_bucket_flags(const double* __restrict__ coef, uint8_t* flags, int64_t n, uint64_t prefix,
                               uint64_t prefix_mask, uint32_t* cand, unsigned long long* n_cand) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        if (!flags[i]) continue;
        const uint64_t b = abs_bits(coef[i]) & prefix_mask;
        if (b > prefix) continue;
        flags[i] = 0;
        if (b == prefix) cand[atomicAdd(n_cand, 1ull)] = (uint32_t)i;
    }
}

// The term limit's cut with every row live: flags[i] = 1 above the threshold
// bucket, 0 in and below it; the bucket's rows are listed as candidates.
__global__ void k_cut_flags(const double* __restrict__ coef, uint8_t* flags, int64_t n, uint64_t prefix,
                            uint64_t prefix_mask, uint32_t* cand, unsigned long long* n_cand) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        const uint64_t b = abs_bits(coef[i]) & prefix_mask;
        flags[i] = b > prefix;
        if (b == prefix) cand[atomicAdd(n_cand, 1ull)] = (uint32_t)i;
    }
}

// Sort keys of the candidates: [~|C| bits, x most significant word first, ..., z ...]:
// ascending order = |C| descending, then canonical key ascending.
template <int W>
__global__ void k_candidate_keys(const uint64_t* __restrict__ rows, const double* __restrict__ coef,
                                 const uint32_t* __restrict__ cand, int64_t k, uint64_t* skeys) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += s) {
        const uint32_t r = cand[i];
        const Key<W> key = load_key<W>(rows, r);
        uint64_t* o = skeys + (size_t)i * (2 * W + 1);
        o[0] = ~abs_bits(coef[r]);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            o[1 + w] = key.x[W - 1 - w];
            o[1 + W + w] = key.z[W - 1 - w];
        }
    }
}

__global__ void k_set_flags_sorted(const uint32_t* __restrict__ cand, const uint32_t* __restrict__ order, int64_t k,
                                   uint8_t* flags) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += s) flags[cand[order[i]]] = 1;
}

// out[i] = keys[order[i] * stride + 0]: the first word of each key, in sorted order.
__global__ void k_gather_word(const uint64_t* __restrict__ keys, int stride, const uint32_t* __restrict__ order,
                              int64_t n, uint64_t* out) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s)
        out[i] = keys[(size_t)order[i] * stride];
}

// Multi-part term limit: the first k candidates in sorted order, each owned
// by the part whose range [offs[p], offs[p + 1]) holds its index, flagged in
// that part's flags.
__global__ void k_set_flags_sorted_parts(const uint32_t* __restrict__ cand, const uint32_t* __restrict__ order,
                                         int64_t k, const int64_t* __restrict__ offs, uint8_t* const* flags,
                                         int n_parts) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += s) {
        const int64_t g = order[i];
        int p = 0;
        while (p + 1 < n_parts && offs[p + 1] <= g) ++p;
        flags[p][cand[g]] = 1;
    }
}

// ---------------------------------------------------------------- DIS ordering

// skeys[g] = [~coarse(|g|), x[Wd-1], ..., x[0]]: ascending order of these words
// is |g| (20 low mantissa bits cleared) descending, then x ascending.
__global__ void k_dis_sort_keys(int Wd, const uint64_t* __restrict__ gkeys, const double* __restrict__ gsum,
                                int64_t G, uint64_t* skeys) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += s) {
        uint64_t a = abs_bits(gsum[g]) & ~((1ull << 20) - 1ull);
        skeys[(size_t)g * (Wd + 1)] = ~a;
        for (int w = 0; w < Wd; ++w) skeys[(size_t)g * (Wd + 1) + 1 + w] = gkeys[(size_t)g * Wd + (Wd - 1 - w)];
    }
}

__global__ void k_dis_export(int W, int Wd, const uint64_t* __restrict__ gkeys, const double* __restrict__ gsum,
                             const uint32_t* __restrict__ perm, const uint32_t* __restrict__ idx, int64_t k,
                             uint64_t* ox, uint64_t* oz, double* og) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += s) {
        const uint32_t g = idx ? idx[perm[i]] : perm[i];
        bool found = false;
        for (int w = 0; w < W; ++w) {
            const uint64_t x = gkeys[(size_t)g * Wd + w];
            ox[(size_t)i * W + w] = x;
            oz[(size_t)i * W + w] = found ? 0ull : (x & (~x + 1ull));
            found |= (x != 0);
        }
        og[i] = gsum[g];
    }
}

int grid_stride_blocks(int64_t n) {
    int64_t want = (n + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)sm_count() * 8;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

}  // namespace

size_t radix_sort_scratch_bytes(int64_t n) {
    // hist [256][nblocks] + orand
    return (size_t)256 * (size_t)n_tiles(n) * sizeof(uint32_t) + 32 * sizeof(unsigned long long) + 256;
}

void launch_iota(uint32_t* p, int64_t n, cudaStream_t s) {
    if (n > 0) {
        k_iota<<<grid_stride_blocks(n), kThreads, 0, s>>>(p, n);
        note_launch();
    }
}

void radix_sort_indirect(const uint64_t* keys, int stride, const SortPlan& plan, uint32_t* perm,
                         uint32_t* perm_alt, int64_t n, uint32_t** result, void* scratch, size_t scratch_bytes,
                         cudaStream_t s) {
    *result = perm;
    if (n <= 1) return;
    const int64_t nb = n_tiles(n);
    uint32_t* hist = (uint32_t*)scratch;
    unsigned long long* orand =
        (unsigned long long*)((char*)scratch + (((size_t)256 * nb * sizeof(uint32_t) + 255) & ~(size_t)255));
    (void)scratch_bytes;
    // constant digits are skipped: OR and AND of each word over all elements
    unsigned long long init[18];
    for (int w = 0; w < stride; ++w) { init[w] = 0ull; init[stride + w] = ~0ull; }
    cudaMemcpyAsync(orand, init, sizeof(unsigned long long) * 2 * stride, cudaMemcpyHostToDevice, s);
    k_word_orand<<<grid_stride_blocks(n), kThreads, 2 * stride * sizeof(unsigned long long), s>>>(keys, stride, perm,
                                                                                                 n, orand); note_launch();
    unsigned long long host_orand[18];
    cudaMemcpyAsync(host_orand, orand, sizeof(unsigned long long) * 2 * stride, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    uint32_t* a = perm;
    uint32_t* b = perm_alt;
    for (int oi = plan.n_order - 1; oi >= 0; --oi) {
        const int word = plan.order[oi];
        const uint64_t varying = host_orand[word] ^ host_orand[stride + word];
        for (int shift = 0; shift < 64; shift += 8) {
            if (((varying >> shift) & 255ull) == 0) continue;
            k_sort_hist<<<(unsigned)nb, kThreads, 0, s>>>(keys, stride, word, shift, a, n, hist, nb); note_launch();
            k_scan_u32<<<1, 1024, 0, s>>>(hist, 256 * nb); note_launch();
            k_sort_scatter<<<(unsigned)nb, kThreads, 0, s>>>(keys, stride, word, shift, a, b, n, hist, nb); note_launch();
            uint32_t* t = a; a = b; b = t;
        }
    }
    *result = a;
}

size_t compact_scratch_bytes(int64_t n) { return (size_t)n_tiles(n) * 2 * sizeof(uint32_t) + 512; }

void launch_compact_rows(int Wd, const uint8_t* flags, const uint64_t* rows_in, const double* c_in,
                         uint64_t* rows_out, double* c_out, int64_t n, void* scratch, unsigned long long* count,
                         cudaStream_t s) {
    if (n <= 0) {
        cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
        return;
    }
    const int64_t nb = n_tiles(n);
    uint32_t* counts = (uint32_t*)scratch;
    uint32_t* offsets = counts + nb;
    k_flag_count<<<(unsigned)nb, kThreads, 0, s>>>(flags, n, counts); note_launch();
    cudaMemcpyAsync(offsets, counts, nb * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    k_scan_u32<<<1, 1024, 0, s>>>(offsets, nb); note_launch();
    k_total<<<1, 1, 0, s>>>(offsets, counts + nb - 1, nb, count); note_launch();
    switch (Wd) {
        case 1: k_compact_scatter<1><<<(unsigned)nb, kThreads, 0, s>>>(flags, rows_in, c_in, rows_out, c_out, n, offsets); note_launch(); break;
        case 2: k_compact_scatter<2><<<(unsigned)nb, kThreads, 0, s>>>(flags, rows_in, c_in, rows_out, c_out, n, offsets); note_launch(); break;
        default: k_compact_scatter<4><<<(unsigned)nb, kThreads, 0, s>>>(flags, rows_in, c_in, rows_out, c_out, n, offsets); note_launch(); break;
    }
}

size_t compact_inplace_scratch_bytes(int64_t n) {
    return ((size_t)((n + kCompactTile - 1) / kCompactTile) + 1) * sizeof(unsigned long long) + 256;
}

void launch_compact_inplace(int Wd, const uint8_t* flags, uint64_t* rows, double* coef, int64_t n, void* scratch,
                            unsigned long long* count, DevCounters* ctr, cudaStream_t s, uint32_t* new_row) {
    const int64_t nt = (n + kCompactTile - 1) / kCompactTile;
    if (n <= 0) {
        cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
        return;
    }
    unsigned long long* state = (unsigned long long*)scratch;
    unsigned int* tile_counter = (unsigned int*)(state + nt);
    cudaMemsetAsync(scratch, 0, (size_t)(nt + 1) * sizeof(unsigned long long), s);
    switch (Wd) {
        case 1:
            k_compact_inplace<1><<<(unsigned)nt, kThreads, 0, s>>>(flags, rows, coef, n, state, tile_counter, count, ctr,
                                                                  new_row);
            break;
        case 2:
            k_compact_inplace<2><<<(unsigned)nt, kThreads, 0, s>>>(flags, rows, coef, n, state, tile_counter, count, ctr,
                                                                  new_row);
            break;
        default:
            k_compact_inplace<4><<<(unsigned)nt, kThreads, 0, s>>>(flags, rows, coef, n, state, tile_counter, count, ctr,
                                                                  new_row);
            break;
    }
    note_launch();
}

void launch_wait_selftest(const unsigned long long* word, DevCounters* ctr, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(word, ctr);
    note_launch();
}

void launch_coarse_digit_hist(const double* g, int64_t G, int shift, uint64_t prefix, uint64_t prefix_mask,
                              unsigned long long* hist, cudaStream_t s) {
    if (G > 0) {
        k_coarse_digit_hist<<<grid_stride_blocks(G), kThreads, 0, s>>>(g, G, shift, prefix, prefix_mask, hist);
        note_launch();
    }
}

void launch_collect_ge(const double* g, int64_t G, uint64_t t, uint32_t* idx, int64_t cap, unsigned long long* count,
                       cudaStream_t s) {
    if (G > 0) {
        k_collect_ge<<<grid_stride_blocks(G), kThreads, 0, s>>>(g, G, t, idx, cap, count);
        note_launch();
    }
}

void launch_dis_sort_keys_sub(int Wd, const uint64_t* gkeys, const double* gsum, const uint32_t* idx, int64_t k,
                              uint64_t* skeys, cudaStream_t s) {
    if (k > 0) {
        k_dis_sort_keys_sub<<<grid_stride_blocks(k), kThreads, 0, s>>>(Wd, gkeys, gsum, idx, k, skeys);
        note_launch();
    }
}

void launch_pack_rows(int W, int Wd, const uint64_t* x, const uint64_t* z, uint64_t* rows, int64_t n, cudaStream_t s,
                      uint64_t hi_mask, unsigned long long* bad) {
    if (n > 0) {
        k_pack_rows<<<grid_stride_blocks(n), kThreads, 0, s>>>(W, Wd, x, z, rows, n, hi_mask, bad);
        note_launch();
    }
}

void launch_unpack_rows(int W, int Wd, const uint64_t* rows, const double* coef, const uint32_t* perm,
                        uint64_t* x, uint64_t* z, double* c, int64_t n, cudaStream_t s) {
    if (n > 0) {
        k_unpack_rows<<<grid_stride_blocks(n), kThreads, 0, s>>>(W, Wd, rows, coef, perm, x, z, c, n);
        note_launch();
    }
}

void launch_sum_runs(int Wd, const uint64_t* rows, const double* coef, const uint32_t* perm, int64_t n,
                     uint8_t* flags, uint64_t* rows_out, double* c_out, cudaStream_t s, bool keep_zeros) {
    if (n <= 0) return;
    int g = grid_stride_blocks(n);
    switch (Wd) {
        case 1: k_sum_runs<1><<<g, kThreads, 0, s>>>(rows, coef, perm, n, flags, rows_out, c_out, keep_zeros); note_launch(); break;
        case 2: k_sum_runs<2><<<g, kThreads, 0, s>>>(rows, coef, perm, n, flags, rows_out, c_out, keep_zeros); note_launch(); break;
        default: k_sum_runs<4><<<g, kThreads, 0, s>>>(rows, coef, perm, n, flags, rows_out, c_out, keep_zeros); note_launch(); break;
    }
}

void launch_order_violations(int Wd, const uint64_t* rows, int64_t n, unsigned long long* count, cudaStream_t s) {
    if (n <= 1) return;
    const int g = grid_stride_blocks(n);
    switch (Wd) {
        case 1: k_order_violations<1><<<g, kThreads, 0, s>>>(rows, n, count); break;
        case 2: k_order_violations<2><<<g, kThreads, 0, s>>>(rows, n, count); break;
        default: k_order_violations<4><<<g, kThreads, 0, s>>>(rows, n, count); break;
    }
    note_launch();
}

void launch_gather_rows(int Wd, const uint64_t* rows, const double* coef, const uint32_t* perm, int64_t n,
                        uint64_t* rows_out, double* c_out, cudaStream_t s) {
    if (n <= 0) return;
    int g = grid_stride_blocks(n);
    switch (Wd) {
        case 1: k_gather_rows<1><<<g, kThreads, 0, s>>>(rows, coef, perm, n, rows_out, c_out); note_launch(); break;
        case 2: k_gather_rows<2><<<g, kThreads, 0, s>>>(rows, coef, perm, n, rows_out, c_out); note_launch(); break;
        default: k_gather_rows<4><<<g, kThreads, 0, s>>>(rows, coef, perm, n, rows_out, c_out); note_launch(); break;
    }
}

void launch_prune_flags(const double* coef, int64_t n, double eps, uint8_t* flags, unsigned long long* count,
                        cudaStream_t s) {
    if (n > 0) {
        k_prune_flags<<<grid_stride_blocks(n), kThreads, 0, s>>>(coef, n, eps, flags, count);
        note_launch();
    }
}

void launch_abs_digit_hist(const double* coef, const uint8_t* flags, int64_t n, int shift, uint64_t prefix,
                           uint64_t prefix_mask, unsigned long long* hist, cudaStream_t s) {
    if (n > 0)
        k_abs_digit_hist<<<grid_stride_blocks(n), kThreads, 0, s>>>(coef, flags, n, shift, prefix, prefix_mask, hist); note_launch();
}

void launch_budget_flags(const double* coef, uint8_t* flags, int64_t n, uint64_t t_bits, uint32_t* tie_idx,
                         unsigned long long* tie_count, cudaStream_t s) {
    if (n > 0) {
        k_budget_flags<<<grid_stride_blocks(n), kThreads, 0, s>>>(coef, flags, n, t_bits, tie_idx, tie_count);
        note_launch();
    }
}

void launch_set_flags(const uint32_t* idx, int64_t k, uint8_t* flags, cudaStream_t s) {
    if (k > 0) {
        k_set_flags<<<grid_stride_blocks(k), kThreads, 0, s>>>(idx, k, flags);
        note_launch();
    }
}

void launch_abs_digit_hist12(const double* coef, const uint8_t* flags, int64_t n, int shift, uint64_t prefix,
                             uint64_t prefix_mask, unsigned long long* hist, cudaStream_t s) {
    if (n > 0) {
        k_abs_digit_hist12<<<grid_stride_blocks(n), kThreads, 0, s>>>(coef, flags, n, shift, prefix, prefix_mask, hist);
        note_launch();
    }
}

void launch_abs_digit_hist12x2(const double* coef, const uint8_t* flags, int64_t n, int shift1, int shift2,
                               unsigned guess, unsigned long long* hist1, unsigned long long* hist2, cudaStream_t s) {
    if (n > 0) {
        k_abs_digit_hist12x2<<<grid_stride_blocks(n), kThreads, 0, s>>>(coef, flags, n, shift1, shift2, guess, hist1,
                                                                        hist2);
        note_launch();
    }
}

void launch_bucket_values(const double* coef, const uint8_t* flags, int64_t n, uint64_t prefix, uint64_t prefix_mask,
                          double* vals, unsigned long long* n_vals, int64_t cap, cudaStream_t s) {
    if (n > 0) {
        k_bucket_values<<<grid_stride_blocks(n), kThreads, 0, s>>>(coef, flags, n, prefix, prefix_mask, vals, n_vals,
                                                                   (unsigned long long)cap);
        note_launch();
    }
}

void launch_boost_rank(const double* coef, const uint8_t* flags, int64_t n, uint64_t t_bits, double boost, double* rank,
                       cudaStream_t s) {
    if (n > 0) {
        k_boost_rank<<<grid_stride_blocks(n), kThreads, 0, s>>>(coef, flags, n, t_bits, boost, rank);
        note_launch();
    }
}

void launch_bucket_flags(const double* coef, uint8_t* flags, int64_t n, uint64_t prefix, uint64_t prefix_mask,
                         uint32_t* cand, unsigned long long* n_cand, cudaStream_t s) {
    if (n > 0) {
        k_bucket_flags<<<grid_stride_blocks(n), kThreads, 0, s>>>(coef, flags, n, prefix, prefix_mask, cand, n_cand);
        note_launch();
    }
}

void launch_cut_flags(const double* coef, uint8_t* flags, int64_t n, uint64_t prefix, uint64_t prefix_mask,
                      uint32_t* cand, unsigned long long* n_cand, cudaStream_t s) {
    if (n > 0) {
        k_cut_flags<<<grid_stride_blocks(n), kThreads, 0, s>>>(coef, flags, n, prefix, prefix_mask, cand, n_cand);
        note_launch();
    }
}

void launch_candidate_keys(int Wd, const uint64_t* rows, const double* coef, const uint32_t* cand, int64_t k,
                           uint64_t* skeys, cudaStream_t s) {
    if (k <= 0) return;
    const int g = grid_stride_blocks(k);
    switch (Wd) {
        case 1: k_candidate_keys<1><<<g, kThreads, 0, s>>>(rows, coef, cand, k, skeys); note_launch(); break;
        case 2: k_candidate_keys<2><<<g, kThreads, 0, s>>>(rows, coef, cand, k, skeys); note_launch(); break;
        default: k_candidate_keys<4><<<g, kThreads, 0, s>>>(rows, coef, cand, k, skeys); note_launch(); break;
    }
}

void launch_set_flags_sorted(const uint32_t* cand, const uint32_t* order, int64_t k, uint8_t* flags, cudaStream_t s) {
    if (k > 0) {
        k_set_flags_sorted<<<grid_stride_blocks(k), kThreads, 0, s>>>(cand, order, k, flags);
        note_launch();
    }
}

void launch_gather_word(const uint64_t* keys, int stride, const uint32_t* order, int64_t n, uint64_t* out,
                        cudaStream_t s) {
    if (n > 0) {
        k_gather_word<<<grid_stride_blocks(n), kThreads, 0, s>>>(keys, stride, order, n, out);
        note_launch();
    }
}

void launch_set_flags_sorted_parts(const uint32_t* cand, const uint32_t* order, int64_t k, const int64_t* offs,
                                   uint8_t* const* flags, int n_parts, cudaStream_t s) {
    if (k > 0) {
        k_set_flags_sorted_parts<<<grid_stride_blocks(k), kThreads, 0, s>>>(cand, order, k, offs, flags, n_parts);
        note_launch();
    }
}

void launch_dis_sort_keys(int Wd, const uint64_t* gkeys, const double* gsum, int64_t G, uint64_t* skeys,
                          cudaStream_t s) {
    if (G > 0) {
        k_dis_sort_keys<<<grid_stride_blocks(G), kThreads, 0, s>>>(Wd, gkeys, gsum, G, skeys);
        note_launch();
    }
}

void launch_dis_export(int W, int Wd, const uint64_t* gkeys, const double* gsum, const uint32_t* perm,
                       const uint32_t* idx, int64_t k, uint64_t* ox, uint64_t* oz, double* og, cudaStream_t s) {
    if (k > 0) {
        k_dis_export<<<grid_stride_blocks(k), kThreads, 0, s>>>(W, Wd, gkeys, gsum, perm, idx, k, ox, oz, og);
        note_launch();
    }
}

}  // namespace iqcc
