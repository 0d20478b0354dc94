// DIS candidates by partition (App. A "Direct Interaction Space"): one
// candidate per distinct non-empty flip set of H, x = the flip set and z =
// its lowest qubit (one Y, odd Y count).  At a z-eigenstate reference the
// gradient of candidate a sees only the strings whose flip set equals a's
// (Eq. 14-15), so it is a sum over the rows of one flip-set group.
//
// The grouping is a partition join, like the dress (k_pairjoin.cu):
//   1. k_flip_hist     rows with a non-empty flip set counted into 2^k bins by
//                      the top bits of the flip set's hash; a scan gives starts.
//   2. k_flip_scatter  each such row's flip set (and, at a z-eigenstate, its
//                      signed contribution +-C_T to its group's gradient) copied
//                      into its bin (records of whole 32-byte sectors).
//   3. k_flip_join     one block per group of consecutive bins: distinct flip
//                      sets found in a shared-memory table, contributions summed
//                      there (a group may hold any number of rows), one (flip
//                      set, sum) per group appended to the output.
// Every pass streams; the only scattered writes are the bin fronts (small
// enough for L2) and the per-block output ranges.
#include <cuda_runtime.h>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;
constexpr int kSlots = 4096;       // distinct flip sets one join block can hold (about 1024 expected)
constexpr int kTarget = 1024;      // rows per join block on average

template <int W>
__device__ __forceinline__ bool has_flips(const Key<W>& t) {
    uint64_t v = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) v |= t.x[j];
    return v != 0;
}

template <int W>
__device__ __forceinline__ uint64_t flip_hash(const uint64_t* x) {
    Key<W> k;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        k.x[j] = x[j];
        k.z[j] = 0;
    }
    return hash_key<W>(k);
}

// Signed contribution of T to the gradient of its flip set's candidate a at a
// z-eigenstate: C_T times the sign of <Omega| T a |Omega> / i (zero when T
// commutes with a).
template <int W>
__device__ __forceinline__ double basis_contribution(const Key<W>& t, double c, const uint64_t* occ) {
    Key<W> a;
    bool found = false;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        a.x[j] = t.x[j];
        a.z[j] = found ? 0ull : (t.x[j] & (~t.x[j] + 1));
        found |= t.x[j] != 0;
    }
    if (!anticommutes<W>(t, a)) return 0.0;
    const Key<W> q = key_xor<W>(t, a);
    const int s = product_sign<W>(t, 1, a, q);
    int odd = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) odd += __popcll(q.z[j] & occ[j]);
    const bool neg = (s < 0) ^ (bool)(odd & 1);
    return neg ? -c : c;
}

template <int W>
struct Occ {
    uint64_t w[W];
};

// A bin record: the flip set (W words), the contribution, the flip set's
// hash, zero padding to whole 32-byte sectors (W = 1, 2: 32 B; W = 4: 64 B),
// so that the scattered writes fill whole sectors.
template <int W>
constexpr int frec_words() { return (W + 2 + 3) / 4 * 4; }

template <int W>
__global__ void __launch_bounds__(kThreads) k_flip_hist(const uint64_t* __restrict__ rows, int64_t M, int shift,
                                                        uint32_t* counts, DevCounters* ctr) {
    unsigned n = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        const Key<W> t = load_key<W>(rows, i);
        if (has_flips<W>(t)) {
            atomicAdd(&counts[flip_hash<W>(t.x) >> shift], 1u);
            ++n;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xFFFFFFFFu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(&ctr->aux, (unsigned long long)n);
}

// cursor[b]: bin start in, bin end out.
template <int W, bool VALUES>
__global__ void __launch_bounds__(kThreads) k_flip_scatter(const uint64_t* __restrict__ rows,
                                                           const double* __restrict__ coef, int64_t M, Occ<W> occ,
                                                           int shift, uint32_t* cursor, uint64_t* rr) {
    constexpr int R = frec_words<W>();
    constexpr int kRows = 4;  // rows per thread and step: their position round trips overlap
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * kRows;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kRows; i0 < M; i0 += stride) {
        Key<W> t[kRows];
        bool f[kRows];
        uint32_t p[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            f[r] = i0 + r < M;
            if (f[r]) {
                t[r] = load_key<W>(rows, i0 + r);
                f[r] = has_flips<W>(t[r]);
            }
            if (f[r]) p[r] = atomicAdd(&cursor[flip_hash<W>(t[r].x) >> shift], 1u);
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            if (!f[r]) continue;
            uint64_t w[R];
#pragma unroll
            for (int j = 0; j < R; ++j) w[j] = 0;
#pragma unroll
            for (int j = 0; j < W; ++j) w[j] = t[r].x[j];
            if (VALUES) w[W] = (uint64_t)__double_as_longlong(basis_contribution<W>(t[r], coef[i0 + r], occ.w));
            w[W + 1] = flip_hash<W>(t[r].x);  // for the join, which would otherwise hash the flip set again
            ulonglong2* d = reinterpret_cast<ulonglong2*>(rr + (size_t)p[r] * R);
#pragma unroll
            for (int j = 0; j < R / 2; ++j) d[j] = make_ulonglong2(w[2 * j], w[2 * j + 1]);
        }
    }
}

// Block j: bins [j*bpb, (j+1)*bpb), rows [start[b0], start[b1]) of the copies.
// A group (one flip set) may hold any number of rows, so the shared-memory
// table bounds the distinct flip sets of a block (kSlots / 2 on average,
// which the bin sizing keeps), not its rows: every slot holds the first row of
// its group (tag and index) and the group's sum.
template <int W, bool VALUES>
__global__ void __launch_bounds__(kThreads) k_flip_join(const uint64_t* __restrict__ rr,
                                                        const uint32_t* __restrict__ start, uint32_t n_bins,
                                                        uint32_t bins_per_block, uint64_t* gkeys, double* gsum,
                                                        int64_t max_groups, DevCounters* ctr) {
    constexpr int R = frec_words<W>();
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* table = reinterpret_cast<unsigned long long*>(smem);  // [kSlots]: tag32 | row32
    double* sum = reinterpret_cast<double*>(table + kSlots);                     // [kSlots]
    __shared__ unsigned int s_count;
    __shared__ unsigned long long s_base;
    const uint32_t b0 = blockIdx.x * bins_per_block;
    const uint32_t b1 = min(b0 + bins_per_block, n_bins);
    const uint32_t r0 = start[b0];
    const int64_t n = (int64_t)start[b1] - r0;
    if (n <= 0) return;
    for (int s = threadIdx.x; s < kSlots; s += blockDim.x) {
        table[s] = kEmptySlot;
        sum[s] = 0.0;
    }
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    volatile unsigned long long* vt = table;
    bool full = false;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        uint64_t x[W];
#pragma unroll
        for (int j = 0; j < W; ++j) x[j] = rr[(size_t)(r0 + i) * R + j];
        const uint64_t h = rr[(size_t)(r0 + i) * R + W + 1];  // the flip set's hash, stored by the scatter
        const unsigned long long mine = (h & 0xFFFFFFFF00000000ull) | (unsigned long long)(uint32_t)i;
        uint32_t s = (uint32_t)h & (kSlots - 1);
        int probe = 0;
        for (; probe < kSlots; ++probe) {
            unsigned long long v = vt[s];
            if (v == kEmptySlot) {
                v = atomicCAS(&table[s], kEmptySlot, mine);
                if (v == kEmptySlot) break;  // first row of its group
            }
            if ((v >> 32) == (h >> 32)) {
                const uint32_t j = (uint32_t)v;
                bool same = true;
#pragma unroll
                for (int w = 0; w < W; ++w) same &= rr[(size_t)(r0 + j) * R + w] == x[w];
                if (same) break;
            }
            s = (s + 1) & (kSlots - 1);
        }
        if (probe == kSlots) {
            full = true;
            continue;
        }
        if (VALUES) atomicAdd(&sum[s], __longlong_as_double((long long)rr[(size_t)(r0 + i) * R + W]));
    }
    if (full) set_error(ctr, IQCC_ERR_HASH_FULL, 80);  // more distinct flip sets than slots in one block
    __syncthreads();
    unsigned cnt = 0;
    for (int s = threadIdx.x; s < kSlots; s += blockDim.x) cnt += table[s] != kEmptySlot;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s_count, cnt);
    __syncthreads();
    if (threadIdx.x == 0) {
        s_base = atomicAdd(&ctr->n_groups, (unsigned long long)s_count);
        s_count = 0;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < kSlots; s += blockDim.x) {
        const unsigned long long v = table[s];
        if (v == kEmptySlot) continue;
        const int64_t g = (int64_t)s_base + (int64_t)atomicAdd(&s_count, 1u);
        if (g >= max_groups) {  // cannot happen: groups <= rows
            set_error(ctr, IQCC_ERR_STATE, 81);
            continue;
        }
        const uint32_t j = (uint32_t)v;
#pragma unroll
        for (int w = 0; w < W; ++w) gkeys[g * W + w] = rr[(size_t)(r0 + j) * R + w];
        gsum[g] = VALUES ? sum[s] : 0.0;
    }
}

size_t join_smem() { return (size_t)kSlots * 8 + (size_t)kSlots * 8; }

int grid_cap(int64_t items, int per_sm) {
    int64_t want = (items + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sm_count() * per_sm;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

template <int W>
void flip_group(const uint64_t* rows, const double* coef, int64_t M, const uint64_t* occ_words, bool values,
                int log2_bins, uint32_t* arr, uint64_t* rr, int64_t n_flip, uint64_t* gkeys, double* gsum,
                int64_t max_groups, DevCounters* ctr, cudaStream_t s) {
    Occ<W> occ{};
    for (int j = 0; j < W; ++j) occ.w[j] = occ_words[j];
    const int shift = 64 - log2_bins;
    const uint32_t NB = 1u << log2_bins;
    const int grid = grid_cap(M, 8);
    if (values) k_flip_scatter<W, true><<<grid, kThreads, 0, s>>>(rows, coef, M, occ, shift, arr + 1, rr);
    else k_flip_scatter<W, false><<<grid, kThreads, 0, s>>>(rows, coef, M, occ, shift, arr + 1, rr);
    uint32_t bpb = 1;  // consecutive bins per block: about kTarget rows
    const double per_bin = (double)n_flip / (double)NB;
    while (bpb < NB && (double)(bpb * 2) * per_bin <= kTarget) bpb *= 2;
    const unsigned blocks = (NB + bpb - 1) / bpb;
    static std::atomic<unsigned long long> attr{0};
    if (first_on_device(&attr)) {
        cudaFuncSetAttribute(k_flip_join<W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)join_smem());
        cudaFuncSetAttribute(k_flip_join<W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)join_smem());
    }
    if (values)
        k_flip_join<W, true><<<blocks, kThreads, join_smem(), s>>>(rr, arr, NB, bpb, gkeys, gsum, max_groups, ctr);
    else
        k_flip_join<W, false><<<blocks, kThreads, join_smem(), s>>>(rr, arr, NB, bpb, gkeys, gsum, max_groups, ctr);
}

}  // namespace

void launch_flip_hist(int Wd, const uint64_t* rows, int64_t M, int log2_bins, uint32_t* counts, DevCounters* ctr,
                      cudaStream_t s) {
    if (M <= 0) return;
    const int grid = grid_cap(M, 8), shift = 64 - log2_bins;
    switch (Wd) {
        case 1: k_flip_hist<1><<<grid, kThreads, 0, s>>>(rows, M, shift, counts, ctr); break;
        case 2: k_flip_hist<2><<<grid, kThreads, 0, s>>>(rows, M, shift, counts, ctr); break;
        default: k_flip_hist<4><<<grid, kThreads, 0, s>>>(rows, M, shift, counts, ctr); break;
    }
    note_launch();
}

size_t flip_record_bytes(int Wd) {
    return 8 * (size_t)(Wd == 1 ? frec_words<1>() : (Wd == 2 ? frec_words<2>() : frec_words<4>()));
}

void launch_flip_group(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* occ_words,
                       bool values, int log2_bins, uint32_t* arr, uint64_t* rr, int64_t n_flip, uint64_t* gkeys,
                       double* gsum, int64_t max_groups, DevCounters* ctr, cudaStream_t s) {
    if (M <= 0 || n_flip <= 0) return;
    switch (Wd) {
        case 1: flip_group<1>(rows, coef, M, occ_words, values, log2_bins, arr, rr, n_flip, gkeys, gsum, max_groups,
                              ctr, s); break;
        case 2: flip_group<2>(rows, coef, M, occ_words, values, log2_bins, arr, rr, n_flip, gkeys, gsum, max_groups,
                              ctr, s); break;
        default: flip_group<4>(rows, coef, M, occ_words, values, log2_bins, arr, rr, n_flip, gkeys, gsum, max_groups,
                               ctr, s); break;
    }
    note_launch(2);
}

}  // namespace iqcc
