// Dressing by pair partition: the merge of Eq. 5 (App. D Eq. 18, "insert if
// unique, else add") without a resident index and without random DRAM access.
//
// A string T that anticommutes with P pairs with exactly one other string,
// its partner Q = T xor P (q -> q xor P is a bijection, and Q anticommutes
// with P as T does).  Both members of a pair have the same pair key: the
// member whose bit at P's lowest set bit is clear (exactly one member has
// that bit clear).  So a partition of the
// anticommuting rows by a hash of their pair key puts both members of every
// present pair in the same partition, and the merge becomes a local join:
//
//   1. k_pair_hist   one pass over the keys: how many anticommuting rows fall
//                    in each of 2^k bins (the top k bits of the pair key's
//                    hash); an exclusive scan turns the counts into bin starts.
//   2. k_pair_split  one pass over the rows: the commuting rows are compacted
//                    in place (stable, decoupled look-back), the anticommuting
//                    ones are copied with their coefficients into their bins.
//   3. k_pair_join   one block per group of consecutive bins: the group's
//                    rows are matched by pair key in a shared-memory table,
//                    each row is written back behind the commuting rows with
//                    C_T cos(tau) - s_T C_Q sin(tau) (partner present, i T P =
//                    s_T Q) or C_T cos(tau) (partner absent), and each row
//                    without a partner appends (Q, s_T C_T sin(tau)).
//
// Every pass streams: the only scattered traffic is the bin cursors (an
// L2-resident array of 4-byte counters) and the bin fronts the split writes
// to.  No per-generator index is built or maintained, so compressing H moves
// rows without any index upkeep.  The appended strings are absent from H by
// construction (a present partner would have been found in the same bin), so
// no duplicate merge is needed.
#include <cuda_runtime.h>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;
constexpr int kSplitTile = 1024;           // rows per split tile (4 per thread)
constexpr int kJoinCap = 4096;             // rows one join block can hold
constexpr int kJoinSlots = 8192;           // its shared-memory table (load <= 1/2)
constexpr uint32_t kJoinEmpty = 0xFFFFFFFFu;
constexpr uint16_t kNoPartner = 0xFFFFu;
constexpr int kJoinTarget = 2048;          // rows per join block on average
constexpr unsigned long long kStAgg = 1ull << 62, kStPrefix = 2ull << 62;
constexpr unsigned long long kStMask = (1ull << 62) - 1;

// One generator for every row.
template <int W>
struct OneGen {
    Gen<W> g;
    __device__ __forceinline__ const Gen<W>& operator()(const Key<W>&) const { return g; }
};

// Batches: the generator of the row's problem (tag in z bits 48..63), from a
// device table; the identity (nothing anticommutes) past the table.
struct ProblemGen {
    const Gen<1>* table;
    int B;
    __device__ __forceinline__ Gen<1> operator()(const Key<1>& t) const {
        const int b = (int)(t.z[0] >> kBatchTagShift);
        if (b < B) return table[b];
        Gen<1> none{};
        return none;
    }
};

template <int W, class G>
__global__ void __launch_bounds__(kThreads) k_pair_hist(const uint64_t* __restrict__ rows, int64_t M, G gen_of,
                                                        int shift, uint32_t* counts, DevCounters* ctr,
                                                        const uint8_t* __restrict__ live) {
    const int lane = threadIdx.x & 31;
    unsigned n_anti = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        if (live && !live[i]) continue;
        const Key<W> t = load_key<W>(rows, i);
        const auto& g = gen_of(t);
        if (anticommutes<W>(t, g.p)) {
            atomicAdd(&counts[pair_hash<W>(t, g.p, g.top_word, g.top_mask) >> shift], 1u);
            ++n_anti;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_anti += __shfl_down_sync(0xFFFFFFFFu, n_anti, o);
    if (lane == 0 && n_anti) atomicAdd(&ctr->n_anti, (unsigned long long)n_anti);
}

// cursor[b]: on entry the start of bin b, on exit its end.  COMPACT: rows
// that commute with their generator are compacted in place, stably (tile
// order by a tile counter, offsets by a decoupled look-back: a tile writes
// only after every earlier tile has read its rows, and below the end of its
// own rows), their count to *total.  SCATTER: rows that anticommute are copied
// (key, coefficient) to their bin.  Warps 1.. copy theirs while warp 0 looks
// back, so the look-back's latency is hidden behind the bin writes.  live
// (may be NULL): rows with live[i] == 0 (dropped by a pending term-limit cut)
// are neither kept nor copied.
template <int W, class G, bool SCATTER>
__device__ __forceinline__ void scatter_rows(const Key<W>* key, const double* c, const bool* anti, const G& gen_of,
                                             int shift, uint32_t* cursor, uint64_t* rk, double* rc) {
    if constexpr (!SCATTER) return;
    uint32_t pos[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {  // the four positions first: their round trips overlap
        if (anti[r]) {
            const auto& g = gen_of(key[r]);
            pos[r] = atomicAdd(&cursor[pair_hash<W>(key[r], g.p, g.top_word, g.top_mask) >> shift], 1u);
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (anti[r]) {
            store_key<W>(rk, pos[r], key[r]);
            rc[pos[r]] = c[r];
        }
    }
}

template <int W, class G, bool COMPACT, bool SCATTER>
__global__ void __launch_bounds__(kThreads) k_pair_split(uint64_t* rows, double* coef, int64_t n, G gen_of, int shift,
                                                         uint32_t* cursor, uint64_t* rk, double* rc,
                                                         unsigned long long* state, unsigned int* tile_counter,
                                                         unsigned long long* total, DevCounters* ctr,
                                                         const uint8_t* __restrict__ live) {
    constexpr int kPer = kSplitTile / kThreads;
    static_assert(kPer == 4, "scatter_rows handles 4 rows per thread");
    __shared__ uint32_t s_w[kThreads / 32];
    __shared__ unsigned int s_tile;
    __shared__ unsigned long long s_prefix;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned int t;
    if (COMPACT) {
        if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
        __syncthreads();
        t = s_tile;
    } else {
        t = blockIdx.x;
    }
    const int64_t base = (int64_t)t * kSplitTile;
    const int64_t wbase = base + (int64_t)wid * (kPer * 32);
    Key<W> key[kPer];
    double c[kPer];
    uint32_t rank[kPer];
    bool keep[kPer], anti[kPer];
    uint32_t wcount = 0;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int64_t i = wbase + (int64_t)r * 32 + lane;
        keep[r] = anti[r] = false;
        if (i < n && (!live || live[i])) {  // rows dropped by a pending cut are neither kept nor copied
            key[r] = load_key<W>(rows, i);
            c[r] = coef[i];
            const auto& g = gen_of(key[r]);
            anti[r] = anticommutes<W>(key[r], g.p);
            keep[r] = !anti[r];
        }
        if (COMPACT) {
            const unsigned b = __ballot_sync(0xFFFFFFFFu, keep[r]);
            rank[r] = wcount + __popc(b & lt);
            wcount += __popc(b);
        }
    }
    if (!COMPACT) {
        scatter_rows<W, G, SCATTER>(key, c, anti, gen_of, shift, cursor, rk, rc);
        return;
    }
    if (lane == 0) s_w[wid] = wcount;
    __syncthreads();
    if (wid == 0) {
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
        unsigned long long prefix = 0;
        int64_t p = (int64_t)t - 1;
        int spins = 0;
        while (p >= 0) {
            const int64_t q = p - lane;
            unsigned long long v2 = kStPrefix;  // before tile 0: a prefix of 0
            if (q >= 0) v2 = *(volatile unsigned long long*)(state + q);
            const unsigned pref = __ballot_sync(0xFFFFFFFFu, (v2 & ~kStMask) == kStPrefix);
            const unsigned zero = __ballot_sync(0xFFFFFFFFu, v2 == 0);
            const int stop = pref ? __ffs(pref) - 1 : 31;
            const unsigned upto = stop == 31 ? 0xFFFFFFFFu : ((2u << stop) - 1u);
            if (zero & upto) {
                if (++spins > ctr->wait_limit) {
                    if (lane == 0) set_error(ctr, IQCC_ERR_TIMEOUT, 71);
                    break;
                }
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
            if (base + kSplitTile >= n) *total = prefix + count;
        }
    } else {
        scatter_rows<W, G, SCATTER>(key, c, anti, gen_of, shift, cursor, rk, rc);
    }
    __syncthreads();
    if (wid == 0) scatter_rows<W, G, SCATTER>(key, c, anti, gen_of, shift, cursor, rk, rc);
    const unsigned long long out = s_prefix + s_w[wid];
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        if (keep[r]) {
            store_key<W>(rows, (int64_t)(out + rank[r]), key[r]);
            coef[out + rank[r]] = c[r];
        }
    }
}

// Block j joins bins [j*bpb, (j+1)*bpb): records [start[b0], start[b1]).
// WRITE: the dressed rows go to rows/coef from *m_comm on (the commuting rows
// end there), each block's at the position it reserves on out_cursor;
// appended partners follow the block's own rows.  Always: the number of rows
// without a partner is added to ctr->n_new.
template <int W, class G, bool WRITE>
__global__ void __launch_bounds__(kThreads) k_pair_join(const uint64_t* __restrict__ rk, const double* __restrict__ rc,
                                                        const uint32_t* __restrict__ start, uint32_t n_bins,
                                                        uint32_t bins_per_block, G gen_of, uint64_t* rows,
                                                        double* coef, const unsigned long long* __restrict__ m_comm,
                                                        unsigned long long* out_cursor, DevCounters* ctr) {
    __shared__ uint32_t table[kJoinSlots];
    __shared__ uint16_t partner[kJoinCap];
    __shared__ unsigned int s_single, s_app;
    __shared__ unsigned long long s_base;
    const uint32_t b0 = blockIdx.x * bins_per_block;
    const uint32_t b1 = min(b0 + bins_per_block, n_bins);
    const uint32_t r0 = start[b0];
    const int n = (int)(start[b1] - r0);
    if (n <= 0) return;
    if (n > kJoinCap) {  // far beyond any statistical fluctuation of a hash partition
        if (threadIdx.x == 0) set_error(ctr, IQCC_ERR_HASH_FULL, 70);
        return;
    }
    for (int s = threadIdx.x; s < kJoinSlots; s += blockDim.x) table[s] = kJoinEmpty;
    for (int s = threadIdx.x; s < n; s += blockDim.x) partner[s] = kNoPartner;
    if (threadIdx.x == 0) {
        s_single = 0;
        s_app = 0;
    }
    __syncthreads();
    // Match by pair key.  Both members of a pair probe the same slot sequence;
    // the first inserts itself at the first empty slot, the second meets it
    // there (every slot before it stays occupied) and links the two.
    volatile uint32_t* vt = table;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Key<W> t = load_key<W>(rk, (int64_t)r0 + i);
        const auto& g = gen_of(t);
        const uint64_t h = pair_hash<W>(t, g.p, g.top_word, g.top_mask);
        const Key<W> q = key_xor<W>(t, g.p);
        const uint32_t tag = (uint32_t)(h >> 16) & 0xFFFF0000u;
        const uint32_t mine = tag | (uint32_t)i;
        uint32_t s = (uint32_t)h & (kJoinSlots - 1);
        for (int probe = 0; probe < kJoinSlots; ++probe) {
            uint32_t v = vt[s];
            if (v == kJoinEmpty) {
                v = atomicCAS(&table[s], kJoinEmpty, mine);
                if (v == kJoinEmpty) break;
            }
            if ((v & 0xFFFF0000u) == tag) {
                const int j = (int)(v & 0xFFFFu);
                if (key_equal<W>(load_key<W>(rk, (int64_t)r0 + j), q)) {
                    partner[i] = (uint16_t)j;
                    partner[j] = (uint16_t)i;
                    break;
                }
            }
            s = (s + 1) & (kJoinSlots - 1);
        }
    }
    __syncthreads();
    unsigned cnt = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) cnt += partner[i] == kNoPartner;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s_single, cnt);
    __syncthreads();
    const unsigned n_single = s_single;
    if (threadIdx.x == 0) {
        if (n_single) atomicAdd(&ctr->n_new, (unsigned long long)n_single);
        if (WRITE) s_base = *m_comm + atomicAdd(out_cursor, (unsigned long long)(n + n_single));
    }
    if (!WRITE) return;
    __syncthreads();
    const int64_t base = (int64_t)s_base;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Key<W> t = load_key<W>(rk, (int64_t)r0 + i);
        const auto& g = gen_of(t);
        const Key<W> q = key_xor<W>(t, g.p);
        const double sg = (double)product_sign<W>(t, g.yP, g.p, q);
        const double ct = rc[r0 + i];
        const int p = partner[i];
        double cn;
        if (p != kNoPartner) {
            cn = ct * g.cos_t - sg * rc[r0 + p] * g.sin_t;
        } else {
            cn = ct * g.cos_t;
            const int64_t r = base + n + (int64_t)atomicAdd(&s_app, 1u);
            store_key<W>(rows, r, q);
            coef[r] = sg * ct * g.sin_t;
        }
        store_key<W>(rows, base + i, t);
        coef[base + i] = cn;
    }
}

int grid_cap(int64_t items, int per_sm) {
    int64_t want = (items + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sm_count() * per_sm;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

// The three launches for one provider type.
template <int W, class G>
struct PairLaunch {
    static void hist(const G& g, const uint64_t* rows, int64_t M, int shift, uint32_t* counts, DevCounters* ctr,
                     const uint8_t* live, cudaStream_t s) {
        k_pair_hist<W, G><<<grid_cap(M, 8), kThreads, 0, s>>>(rows, M, g, shift, counts, ctr, live);
    }
    static void split(const G& g, bool compact, bool scatter, uint64_t* rows, double* coef, int64_t M, int shift,
                      uint32_t* cursor, uint64_t* rk, double* rc, unsigned long long* state,
                      unsigned int* tile_counter, unsigned long long* total, DevCounters* ctr, const uint8_t* live,
                      cudaStream_t s) {
        const unsigned nt = (unsigned)((M + kSplitTile - 1) / kSplitTile);
        if (compact && scatter)
            k_pair_split<W, G, true, true><<<nt, kThreads, 0, s>>>(rows, coef, M, g, shift, cursor, rk, rc, state,
                                                                    tile_counter, total, ctr, live);
        else if (compact)
            k_pair_split<W, G, true, false><<<nt, kThreads, 0, s>>>(rows, coef, M, g, shift, cursor, rk, rc, state,
                                                                     tile_counter, total, ctr, live);
        else
            k_pair_split<W, G, false, true><<<nt, kThreads, 0, s>>>(rows, coef, M, g, shift, cursor, rk, rc, state,
                                                                     tile_counter, total, ctr, live);
    }
    static void join(const G& g, bool write, const uint64_t* rk, const double* rc, const uint32_t* start, uint32_t n_bins,
                     uint32_t bpb, uint64_t* rows, double* coef, const unsigned long long* m_comm,
                     unsigned long long* out_cursor, DevCounters* ctr, cudaStream_t s) {
        const unsigned blocks = (n_bins + bpb - 1) / bpb;
        if (write)
            k_pair_join<W, G, true><<<blocks, kThreads, 0, s>>>(rk, rc, start, n_bins, bpb, g, rows, coef, m_comm,
                                                                 out_cursor, ctr);
        else
            k_pair_join<W, G, false><<<blocks, kThreads, 0, s>>>(rk, rc, start, n_bins, bpb, g, rows, coef, m_comm,
                                                                  out_cursor, ctr);
    }
};

// Calls f(launcher, provider) with the launcher type and generator provider of the dress.
template <class F>
void with_provider(const PairDress& d, F&& f) {
    if (d.gens) {
        f(PairLaunch<1, ProblemGen>{}, ProblemGen{d.gens, d.B});
        return;
    }
    switch (d.Wd) {
        case 1: f(PairLaunch<1, OneGen<1>>{}, OneGen<1>{make_gen<1>(d.pkey, d.cos_t, d.sin_t)}); break;
        case 2: f(PairLaunch<2, OneGen<2>>{}, OneGen<2>{make_gen<2>(d.pkey, d.cos_t, d.sin_t)}); break;
        default: f(PairLaunch<4, OneGen<4>>{}, OneGen<4>{make_gen<4>(d.pkey, d.cos_t, d.sin_t)}); break;
    }
}

}  // namespace

// At most 2048 anticommuting rows per bin on average (every row of H
// anticommuting), at least 1024 bins.  Few enough bins that the split's bin
// fronts (a key sector and a coefficient sector each) stay in L2, where the
// 8-byte coefficient writes of one bin merge into whole sectors.
int pair_bins_log2(int64_t M) {
    int k = 10;
    while (k < 31 && ((int64_t)1 << k) * kJoinTarget < M) ++k;
    return k;
}

uint32_t pair_bins_per_block(int64_t n_anti, int log2_bins) {
    const double per_bin = (double)n_anti / (double)((int64_t)1 << log2_bins);
    uint32_t bpb = 1;
    while (bpb < (1u << log2_bins) && (double)(bpb * 2) * per_bin <= kJoinTarget) bpb *= 2;
    return bpb;
}

size_t pair_split_scratch_bytes(int64_t M) {
    return ((size_t)((M + kSplitTile - 1) / kSplitTile) + 1) * sizeof(unsigned long long) + 256;
}

void launch_pair_hist(const PairDress& d, const uint64_t* rows, int64_t M, int log2_bins, uint32_t* counts,
                      DevCounters* ctr, cudaStream_t s, const uint8_t* live) {
    if (M <= 0) return;
    with_provider(d, [&](auto L, auto g) { decltype(L)::hist(g, rows, M, 64 - log2_bins, counts, ctr, live, s); });
    note_launch();
}

void launch_pair_split(const PairDress& d, bool compact, bool scatter, uint64_t* rows, double* coef, int64_t M,
                       int log2_bins, uint32_t* cursor, uint64_t* rk, double* rc, void* tile_scratch,
                       unsigned long long* m_comm, DevCounters* ctr, cudaStream_t s, const uint8_t* live) {
    if (M <= 0 || !(compact || scatter)) return;
    const int64_t nt = (M + kSplitTile - 1) / kSplitTile;
    unsigned long long* state = (unsigned long long*)tile_scratch;
    unsigned int* tile_counter = (unsigned int*)(state + nt);
    if (compact) cudaMemsetAsync(tile_scratch, 0, (size_t)(nt + 1) * sizeof(unsigned long long), s);
    with_provider(d, [&](auto L, auto g) {
        decltype(L)::split(g, compact, scatter, rows, coef, M, 64 - log2_bins, cursor, rk, rc, state, tile_counter,
                           m_comm, ctr, live, s);
    });
    note_launch();
}

void launch_pair_join(const PairDress& d, bool write, const uint64_t* rk, const double* rc, const uint32_t* start,
                      int log2_bins, uint32_t bins_per_block, uint64_t* rows, double* coef,
                      const unsigned long long* m_comm, unsigned long long* out_cursor, DevCounters* ctr,
                      cudaStream_t s) {
    const uint32_t n_bins = 1u << log2_bins;
    with_provider(d, [&](auto L, auto g) {
        decltype(L)::join(g, write, rk, rc, start, n_bins, bins_per_block, rows, coef, m_comm, out_cursor, ctr, s);
    });
    note_launch();
}

}  // namespace iqcc
