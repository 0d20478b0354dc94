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
//                    hash), and how many commuting rows each tile of 1024 rows
//                    holds; exclusive scans turn both into starts.
//   2. k_pair_split  one pass over the rows into the other row buffer: the
//                    commuting rows are copied to offsets known per tile (the
//                    counting pass counted them), the anticommuting ones with
//                    their coefficients into their bins.
//   3. k_pair_join   one block per group of consecutive bins: the group's
//                    rows are matched by pair key in a shared-memory table,
//                    each row is written behind the commuting rows with
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

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;
constexpr int kJoinCap = 4096;             // rows one join block can hold
constexpr int kJoinSlots = 8192;           // its shared-memory table (load <= 1/2)
constexpr uint32_t kJoinEmpty = 0xFFFFFFFFu;
constexpr uint16_t kNoPartner = 0xFFFFu;
constexpr int kJoinTarget = 2048;          // rows per join block on average

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
                                                        int shift, uint32_t* counts, uint32_t* tile_kept,
                                                        DevCounters* ctr, const uint8_t* __restrict__ live) {
    unsigned n_anti = 0;
    const int64_t n_tiles = (M + kDressTile - 1) / kDressTile;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        constexpr int kPer = kDressTile / kThreads;  // the tile's rows of this thread in flight together
        bool v[kPer], k[kPer];
        Key<W> t[kPer];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int64_t i = tile * kDressTile + r * kThreads + threadIdx.x;
            v[r] = i < M && (!live || live[i]);
        }
#pragma unroll
        for (int r = 0; r < kPer; ++r)
            if (v[r]) t[r] = load_key<W>(rows, tile * kDressTile + r * kThreads + threadIdx.x);
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            k[r] = false;
            if (!v[r]) continue;
            const auto& g = gen_of(t[r]);
            if (anticommutes<W>(t[r], g.p)) {
                atomicAdd(&counts[pair_hash<W>(t[r], g.p, g.top_word, g.top_mask) >> shift], 1u);
                ++n_anti;
            } else {
                k[r] = true;
            }
        }
        int kept = 0;
#pragma unroll
        for (int r = 0; r < kPer; ++r) kept += __syncthreads_count(k[r]);
        if (threadIdx.x == 0) tile_kept[tile] = (uint32_t)kept;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_anti += __shfl_down_sync(0xFFFFFFFFu, n_anti, o);
    if ((threadIdx.x & 31) == 0 && n_anti) atomicAdd(&ctr->n_anti, (unsigned long long)n_anti);
}

// The split, one 1024-row tile per block, from the rows into the other row
// buffer: COMPACT copies the rows that commute with their generator to
// rows_out / coef_out from tile_off[t] on (the counting pass that preceded
// this one counted them per tile, and the offsets are the exclusive scan of
// those counts, so no block waits on another); SCATTER copies the
// anticommuting rows (key, coefficient) to their bins, their positions taken
// first so that the round trips of the four positions of a thread overlap
// with the ranking of the kept rows.  cap == 0: cursor[b] is the start of
// bin b on entry (an exclusive scan of exact counts), its end on exit.
// cap > 0: bins of cap rows each (bin b at [b cap, (b + 1) cap)), cursor
// zeroed on entry and holding the rows that came to each bin on exit; rows
// past a full bin are counted in ctr->aux and not copied.  live (may be
// NULL): rows with live[i] == 0 (dropped by a pending term-limit cut) are
// neither kept nor copied.
template <int W, class G, bool COMPACT, bool SCATTER>
__global__ void __launch_bounds__(kThreads, (W <= 2 ? 4 : 1)) k_pair_split(const uint64_t* __restrict__ rows,
                                                         const double* __restrict__ coef, int64_t n, G gen_of,
                                                         int shift, uint32_t* cursor, uint32_t cap, uint64_t* rk,
                                                         double* rc, const uint32_t* __restrict__ tile_off,
                                                         uint64_t* rows_out, double* coef_out,
                                                         const uint8_t* __restrict__ live, DevCounters* ctr) {
    constexpr int kPer = kDressTile / kThreads;
    __shared__ uint32_t s_w[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t t = blockIdx.x;
    const int64_t wbase = t * kDressTile + (int64_t)wid * (kPer * 32);
    const uint32_t off0 = COMPACT ? tile_off[t] : 0u;  // loaded with the rows
    Key<W> key[kPer];
    double c[kPer];
    uint32_t rank[kPer], pos[kPer];
    bool keep[kPer], anti[kPer];
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int64_t i = wbase + (int64_t)r * 32 + lane;
        keep[r] = anti[r] = false;
        if (i < n && (!live || live[i])) {
            key[r] = load_key<W>(rows, i);
            c[r] = coef[i];
        }
    }
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int64_t i = wbase + (int64_t)r * 32 + lane;
        if (i < n && (!live || live[i])) {
            const auto& g = gen_of(key[r]);
            anti[r] = anticommutes<W>(key[r], g.p);
            keep[r] = !anti[r];
            if (SCATTER && anti[r]) {
                const uint32_t bin = (uint32_t)(pair_hash<W>(key[r], g.p, g.top_word, g.top_mask) >> shift);
                pos[r] = atomicAdd(&cursor[bin], 1u);
                if (cap) {  // fixed-size bins: the bin's slot, or an overflow (the caller redoes the dress)
                    if (pos[r] < cap) {
                        pos[r] += bin * cap;
                    } else {
                        anti[r] = false;
                        atomicAdd(&ctr->aux, 1ull);
                    }
                }
            }
        }
    }
    if (COMPACT) {
        uint32_t wcount = 0;
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const unsigned b = __ballot_sync(0xFFFFFFFFu, keep[r]);
            rank[r] = wcount + __popc(b & lt);
            wcount += __popc(b);
        }
        if (lane == 0) s_w[wid] = wcount;
        __syncthreads();
        uint32_t off = off0;
        for (int w = 0; w < wid; ++w) off += s_w[w];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            if (keep[r]) {
                store_key<W>(rows_out, (int64_t)(off + rank[r]), key[r]);
                coef_out[off + rank[r]] = c[r];
            }
        }
    }
    if (SCATTER) {
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            if (anti[r]) {
                store_key<W>(rk, pos[r], key[r]);
                rc[pos[r]] = c[r];
            }
        }
    }
}

// Where the join's local row i lives in the bin copies: one contiguous range
// (exact bins), or up to kMaxGroupBins fixed-size bins (range k holds local
// rows [pre[k], pre[k + 1]) from base[k] on).
constexpr int kMaxGroupBins = 4;
struct BinRows {
    uint32_t base[kMaxGroupBins];
    uint32_t pre[kMaxGroupBins + 1];
    int nb;
    __device__ __forceinline__ int64_t operator()(int i) const {
        int k = 0;
#pragma unroll
        for (int q = 1; q < kMaxGroupBins; ++q) k += (q < nb && (uint32_t)i >= pre[q]) ? 1 : 0;
        return (int64_t)base[k] + ((uint32_t)i - pre[k]);
    }
};

// Matches the n rows rk[at(0)], ..., rk[at(n - 1)] by pair key in a shared-memory table:
// partner[i] = j for the two members of a present pair, kNoPartner otherwise.
// Both members of a pair probe the same slot sequence; the first inserts
// itself at the first empty slot, the second meets it there (every slot
// before it stays occupied) and links the two.  table (kJoinSlots, all
// kJoinEmpty) and partner (all kNoPartner) are initialised by the caller.
template <int W, class G>
__device__ __forceinline__ void pair_match(const uint64_t* __restrict__ rk, const BinRows& at, int n,
                                           const G& gen_of, uint32_t* table, uint16_t* partner,
                                           uint32_t smask = kJoinSlots - 1) {
    volatile uint32_t* vt = table;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Key<W> t = load_key<W>(rk, at(i));
        const auto& g = gen_of(t);
        const uint64_t h = pair_hash<W>(t, g.p, g.top_word, g.top_mask);
        const Key<W> q = key_xor<W>(t, g.p);
        const uint32_t tag = (uint32_t)(h >> 16) & 0xFFFF0000u;
        const uint32_t mine = tag | (uint32_t)i;
        uint32_t s = (uint32_t)h & smask;
        for (uint32_t probe = 0; probe <= smask; ++probe) {
            uint32_t v = vt[s];
            if (v == kJoinEmpty) {
                v = atomicCAS(&table[s], kJoinEmpty, mine);
                if (v == kJoinEmpty) break;
            }
            if ((v & 0xFFFF0000u) == tag) {
                const int j = (int)(v & 0xFFFFu);
                if (key_equal<W>(load_key<W>(rk, at(j)), q)) {
                    partner[i] = (uint16_t)j;
                    partner[j] = (uint16_t)i;
                    break;
                }
            }
            s = (s + 1) & smask;
        }
    }
}

// Block j joins bins [j*bpb, (j+1)*bpb): records [start[b0], start[b1]);
// with cap > 0 (fixed-size bins, bpb <= kMaxGroupBins) the records
// [b cap, b cap + min(start[b], cap)) of each of its bins.
// WRITE: the dressed rows go to rows/coef from *kept on (the commuting rows
// end there), each block's at the position it reserves on out_cursor;
// appended partners follow the block's own rows.  Always: the number of rows
// without a partner is added to ctr->n_new.
template <int W, class G, bool WRITE>
__global__ void __launch_bounds__(kThreads) k_pair_join(const uint64_t* __restrict__ rk, const double* __restrict__ rc,
                                                        const uint32_t* __restrict__ start, uint32_t n_bins,
                                                        uint32_t bins_per_block, G gen_of, uint64_t* rows,
                                                        double* coef, const uint32_t* __restrict__ kept,
                                                        unsigned long long* out_cursor, DevCounters* ctr,
                                                        uint32_t cap) {
    __shared__ uint32_t table[kJoinSlots];
    __shared__ uint16_t partner[kJoinCap];
    __shared__ unsigned int s_single, s_app;
    __shared__ unsigned long long s_base;
    BinRows at;
    int n = 0;
    const uint32_t b0 = blockIdx.x * bins_per_block;
    const uint32_t b1 = min(b0 + bins_per_block, n_bins);
    if (cap) {  // fixed-size bins (at most kMaxGroupBins): start[] holds the rows each bin received
        at.nb = (int)(b1 - b0);
        for (int k = 0; k < kMaxGroupBins; ++k) {
            const uint32_t b = b0 + (uint32_t)k;
            at.pre[k] = (uint32_t)n;
            at.base[k] = b * cap;
            if (k < at.nb) n += (int)min(start[b], cap);
        }
        at.pre[kMaxGroupBins] = (uint32_t)n;
    } else {
        at.nb = 1;
        at.base[0] = start[b0];
        at.pre[0] = 0;
        n = (int)(start[b1] - start[b0]);
        for (int k = 1; k <= kMaxGroupBins; ++k) at.pre[k] = (uint32_t)n;
    }
    if (n <= 0) return;
    if (n > kJoinCap) {  // far beyond any statistical fluctuation of a hash partition
        if (threadIdx.x == 0) set_error(ctr, IQCC_ERR_HASH_FULL, 70);
        return;
    }
    uint32_t slots = 64;  // a table of at least four times the rows (up to kJoinSlots), cleared only that far
    while (slots < 4u * (uint32_t)n && slots < (uint32_t)kJoinSlots) slots *= 2;
    for (uint32_t s = threadIdx.x; s < slots; s += blockDim.x) table[s] = kJoinEmpty;
    for (int s = threadIdx.x; s < n; s += blockDim.x) partner[s] = kNoPartner;
    if (threadIdx.x == 0) {
        s_single = 0;
        s_app = 0;
    }
    __syncthreads();
    pair_match<W>(rk, at, n, gen_of, table, partner, slots - 1);
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
        if (WRITE) s_base = (unsigned long long)*kept + atomicAdd(out_cursor, (unsigned long long)(n + n_single));
    }
    if (!WRITE) return;
    __syncthreads();
    const int64_t base = (int64_t)s_base;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Key<W> t = load_key<W>(rk, at(i));
        const auto& g = gen_of(t);
        const Key<W> q = key_xor<W>(t, g.p);
        const double sg = (double)product_sign<W>(t, g.yP, g.p, q);
        const double ct = rc[at(i)];
        const int p = partner[i];
        double cn;
        if (p != kNoPartner) {
            cn = ct * g.cos_t - sg * rc[at(p)] * g.sin_t;
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

// Which of two partitions a key belongs to: partition 0 holds the keys whose
// bits under the partition masks equal aval, partition 1 every other key.
template <int W>
struct TwoParts {
    Key<W> mask, aval;
    uint64_t* rows[2];
    double* coef[2];
    const uint32_t* kept[2];        // rows each partition's split kept (its output starts there)
    unsigned long long* cursor[2];  // zeroed; rows each partition receives from the join
    __device__ __forceinline__ int owner(const Key<W>& k) const {
        uint64_t d = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) d |= ((k.x[j] & mask.x[j]) ^ aval.x[j]) | ((k.z[j] & mask.z[j]) ^ aval.z[j]);
        return d != 0;
    }
};

// As k_pair_join (WRITE), for bins filled from two partitions of one
// Hamiltonian: every output row goes to the partition that owns its key (a
// rotated row stays where it came from; an appended partner T xor P goes to
// its own partition, the other one when P flips the partition bits).  Each
// block counts its outputs per partition, reserves both ranges, and places
// its rows through shared-memory counters.
template <int W, class G>
__global__ void __launch_bounds__(kThreads) k_pair_join2(const uint64_t* __restrict__ rk, const double* __restrict__ rc,
                                                         const uint32_t* __restrict__ start, uint32_t n_bins,
                                                         uint32_t bins_per_block, G gen_of, TwoParts<W> o,
                                                         DevCounters* ctr) {
    __shared__ uint32_t table[kJoinSlots];
    __shared__ uint16_t partner[kJoinCap];
    __shared__ unsigned int s_cnt[2], s_cur[2], s_single;
    __shared__ unsigned long long s_base[2];
    const uint32_t b0 = blockIdx.x * bins_per_block;
    const uint32_t b1 = min(b0 + bins_per_block, n_bins);
    const uint32_t r0 = start[b0];
    const int n = (int)(start[b1] - r0);
    if (n <= 0) return;
    if (n > kJoinCap) {
        if (threadIdx.x == 0) set_error(ctr, IQCC_ERR_HASH_FULL, 71);
        return;
    }
    for (int s = threadIdx.x; s < kJoinSlots; s += blockDim.x) table[s] = kJoinEmpty;
    for (int s = threadIdx.x; s < n; s += blockDim.x) partner[s] = kNoPartner;
    if (threadIdx.x < 2) {
        s_cnt[threadIdx.x] = 0;
        s_cur[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) s_single = 0;
    __syncthreads();
    BinRows at;
    at.nb = 1;
    at.base[0] = r0;
    for (int k = 0; k <= kMaxGroupBins; ++k) at.pre[k] = k ? (uint32_t)n : 0u;
    pair_match<W>(rk, at, n, gen_of, table, partner);
    __syncthreads();
    unsigned c[2] = {0, 0}, single = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Key<W> t = load_key<W>(rk, (int64_t)r0 + i);
        ++c[o.owner(t)];
        if (partner[i] == kNoPartner) {
            ++single;
            ++c[o.owner(key_xor<W>(t, gen_of(t).p))];
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        c[0] += __shfl_down_sync(0xFFFFFFFFu, c[0], off);
        c[1] += __shfl_down_sync(0xFFFFFFFFu, c[1], off);
        single += __shfl_down_sync(0xFFFFFFFFu, single, off);
    }
    if ((threadIdx.x & 31) == 0) {
        if (c[0]) atomicAdd(&s_cnt[0], c[0]);
        if (c[1]) atomicAdd(&s_cnt[1], c[1]);
        if (single) atomicAdd(&s_single, single);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_single) atomicAdd(&ctr->n_new, (unsigned long long)s_single);
        for (int d = 0; d < 2; ++d)
            s_base[d] = (unsigned long long)*o.kept[d] + atomicAdd(o.cursor[d], (unsigned long long)s_cnt[d]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Key<W> t = load_key<W>(rk, (int64_t)r0 + i);
        const auto& g = gen_of(t);
        const Key<W> q = key_xor<W>(t, g.p);
        const double sg = (double)product_sign<W>(t, g.yP, g.p, q);
        const double ct = rc[r0 + i];
        const int p = partner[i];
        const int dt = o.owner(t);
        const int64_t rt = (int64_t)s_base[dt] + atomicAdd(&s_cur[dt], 1u);
        if (p != kNoPartner) {
            store_key<W>(o.rows[dt], rt, t);
            o.coef[dt][rt] = ct * g.cos_t - sg * rc[r0 + p] * g.sin_t;
        } else {
            store_key<W>(o.rows[dt], rt, t);
            o.coef[dt][rt] = ct * g.cos_t;
            const int dq = o.owner(q);
            const int64_t rq = (int64_t)s_base[dq] + atomicAdd(&s_cur[dq], 1u);
            store_key<W>(o.rows[dq], rq, q);
            o.coef[dq][rq] = sg * ct * g.sin_t;
        }
    }
}

// ---------------------------------------------------------------------------
// Load of rows in any order: repeated keys summed (Eq. 2: one coefficient per
// distinct string) by the same partition-and-join scheme, keyed on the whole
// key.  k_key_hist counts rows per bin (top L bits of the key's hash),
// k_key_split copies each row with its input index into its bin, and
// k_key_join matches equal keys of a bin group in shared memory; each group
// of equal keys sums its coefficients in input order (so the result equals a
// stable sort followed by run sums), and the distinct keys with a non-zero
// sum are written out in bin order.

template <int W>
__global__ void __launch_bounds__(kThreads) k_key_hist(const uint64_t* __restrict__ rows, int64_t n, int shift,
                                                       uint32_t* counts) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s)
        atomicAdd(&counts[hash_key<W>(load_key<W>(rows, i)) >> shift], 1u);
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_key_split(const uint64_t* __restrict__ rows,
                                                        const double* __restrict__ coef, int64_t n, int shift,
                                                        uint32_t* cursor, uint64_t* rk, double* rc, uint32_t* ri) {
    constexpr int kPer = 4;
    const int64_t base = ((int64_t)blockIdx.x * kPer) * blockDim.x + threadIdx.x;
    Key<W> key[kPer];
    uint32_t pos[kPer];
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int64_t i = base + (int64_t)r * blockDim.x;
        if (i < n) {
            key[r] = load_key<W>(rows, i);
            pos[r] = atomicAdd(&cursor[hash_key<W>(key[r]) >> shift], 1u);
        }
    }
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int64_t i = base + (int64_t)r * blockDim.x;
        if (i < n) {
            store_key<W>(rk, pos[r], key[r]);
            rc[pos[r]] = coef[i];
            ri[pos[r]] = (uint32_t)i;
        }
    }
}

// The sum of the group headed by row h (its other members linked from
// lst[h] through nxt) in ascending input index.
__device__ __forceinline__ double key_group_sum(int h, const uint32_t* lst, const uint16_t* nxt,
                                                const uint32_t* __restrict__ ri, const double* __restrict__ rc,
                                                uint32_t r0) {
    if (lst[h] == kJoinEmpty) return rc[r0 + h];
    double sum = 0.0;
    uint32_t last = 0;
    bool first = true;
    for (;;) {  // repeatedly the smallest input index above the last one taken
        int best = -1;
        uint32_t bi = 0xFFFFFFFFu;
        int m = h;
        uint32_t link = lst[h];
        for (;;) {
            const uint32_t v = ri[r0 + m];
            if ((first || v > last) && v < bi) {
                bi = v;
                best = m;
            }
            if (link == kJoinEmpty) break;
            m = (int)link;
            link = nxt[m] == kNoPartner ? kJoinEmpty : (uint32_t)nxt[m];
        }
        if (best < 0) break;
        sum += rc[r0 + best];
        last = bi;
        first = false;
    }
    return sum;
}

constexpr size_t kKeyJoinSmem = sizeof(uint32_t) * kJoinSlots + sizeof(uint16_t) * kJoinCap +
                                sizeof(uint32_t) * kJoinCap + sizeof(uint16_t) * kJoinCap;

// Block j: bins [j*bpb, (j+1)*bpb), rows [start[b0], start[b1]) (at most
// kJoinCap: the caller checks the groups first; a larger one is an error).
// Writes the distinct keys with non-zero sums to rows_out / c_out at
// positions reserved on out_cursor.
template <int W>
__global__ void __launch_bounds__(kThreads) k_key_join(const uint64_t* __restrict__ rk, const double* __restrict__ rc,
                                                       const uint32_t* __restrict__ ri,
                                                       const uint32_t* __restrict__ start, uint32_t n_bins,
                                                       uint32_t bins_per_block, uint64_t* rows_out, double* c_out,
                                                       unsigned long long* out_cursor, DevCounters* ctr) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint32_t* table = reinterpret_cast<uint32_t*>(s_dyn);
    uint32_t* lst = table + kJoinSlots;
    uint16_t* head = reinterpret_cast<uint16_t*>(lst + kJoinCap);
    uint16_t* nxt = head + kJoinCap;
    __shared__ unsigned int s_cnt, s_cur;
    __shared__ unsigned long long s_base;
    const uint32_t b0 = blockIdx.x * bins_per_block;
    const uint32_t b1 = min(b0 + bins_per_block, n_bins);
    const uint32_t r0 = start[b0];
    const int n = (int)(start[b1] - r0);
    if (n <= 0) return;
    if (n > kJoinCap) {
        if (threadIdx.x == 0) set_error(ctr, IQCC_ERR_HASH_FULL, 72);
        return;
    }
    for (int s = threadIdx.x; s < kJoinSlots; s += blockDim.x) table[s] = kJoinEmpty;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        lst[s] = kJoinEmpty;
        nxt[s] = kNoPartner;
    }
    if (threadIdx.x == 0) {
        s_cnt = 0;
        s_cur = 0;
    }
    __syncthreads();
    // every row finds the first row that claimed its key's slot (its group's head)
    volatile uint32_t* vt = table;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Key<W> t = load_key<W>(rk, (int64_t)r0 + i);
        const uint64_t h = hash_key<W>(t);
        const uint32_t tag = (uint32_t)(h >> 16) & 0xFFFF0000u;
        uint32_t s = (uint32_t)h & (kJoinSlots - 1);
        int hd = i;
        for (int probe = 0; probe < kJoinSlots; ++probe) {
            uint32_t v = vt[s];
            if (v == kJoinEmpty) {
                v = atomicCAS(&table[s], kJoinEmpty, tag | (uint32_t)i);
                if (v == kJoinEmpty) break;  // i heads its key's group
            }
            if ((v & 0xFFFF0000u) == tag) {
                const int j = (int)(v & 0xFFFFu);
                if (key_equal<W>(load_key<W>(rk, (int64_t)r0 + j), t)) {
                    hd = j;
                    break;
                }
            }
            s = (s + 1) & (kJoinSlots - 1);
        }
        head[i] = (uint16_t)hd;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {  // the other members hang off their head
        const int h = head[i];
        if (h != i) {
            const uint32_t old = atomicExch(&lst[h], (uint32_t)i);
            nxt[i] = old == kJoinEmpty ? kNoPartner : (uint16_t)old;
        }
    }
    __syncthreads();
    unsigned cnt = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (head[i] == i && key_group_sum(i, lst, nxt, ri, rc, r0) != 0.0) ++cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (threadIdx.x == 0) s_base = atomicAdd(out_cursor, (unsigned long long)s_cnt);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (head[i] != i) continue;
        const double v = key_group_sum(i, lst, nxt, ri, rc, r0);
        if (v == 0.0) continue;
        const int64_t q = (int64_t)s_base + atomicAdd(&s_cur, 1u);
        store_key<W>(rows_out, q, load_key<W>(rk, (int64_t)r0 + i));
        c_out[q] = v;
    }
}

// Rows flagged in each tile of kDressTile rows (flags only): tile_kept[t].
__global__ void __launch_bounds__(kThreads) k_flag_tiles(const uint8_t* __restrict__ flags, int64_t n,
                                                         uint32_t* tile_kept) {
    constexpr int kPer = kDressTile / kThreads;
    const int64_t base = (int64_t)blockIdx.x * kDressTile;
    bool f[kPer];
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int64_t i = base + r * kThreads + threadIdx.x;
        f[r] = i < n && flags[i];
    }
    int kept = 0;
#pragma unroll
    for (int r = 0; r < kPer; ++r) kept += __syncthreads_count(f[r]);
    if (threadIdx.x == 0) tile_kept[blockIdx.x] = (uint32_t)kept;
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
    static void hist(const G& g, const uint64_t* rows, int64_t M, int shift, uint32_t* counts, uint32_t* tile_kept,
                     DevCounters* ctr, const uint8_t* live, cudaStream_t s) {
        const int64_t n_tiles = (M + kDressTile - 1) / kDressTile;
        const int grid = (int)std::min<int64_t>(n_tiles, (int64_t)sm_count() * 8);
        k_pair_hist<W, G><<<grid, kThreads, 0, s>>>(rows, M, g, shift, counts, tile_kept, ctr, live);
    }
    static void split(const G& g, bool compact, bool scatter, const uint64_t* rows, const double* coef, int64_t M,
                      int shift, uint32_t* cursor, uint32_t cap, uint64_t* rk, double* rc, const uint32_t* tile_off,
                      uint64_t* rows_out, double* coef_out, const uint8_t* live, DevCounters* ctr, cudaStream_t s) {
        const unsigned nt = (unsigned)((M + kDressTile - 1) / kDressTile);
        if (compact && scatter)
            k_pair_split<W, G, true, true><<<nt, kThreads, 0, s>>>(rows, coef, M, g, shift, cursor, cap, rk, rc,
                                                                    tile_off, rows_out, coef_out, live, ctr);
        else if (compact)
            k_pair_split<W, G, true, false><<<nt, kThreads, 0, s>>>(rows, coef, M, g, shift, cursor, cap, rk, rc,
                                                                     tile_off, rows_out, coef_out, live, ctr);
        else
            k_pair_split<W, G, false, true><<<nt, kThreads, 0, s>>>(rows, coef, M, g, shift, cursor, cap, rk, rc,
                                                                     tile_off, rows_out, coef_out, live, ctr);
    }
    static void join(const G& g, bool write, const uint64_t* rk, const double* rc, const uint32_t* start,
                     uint32_t n_bins, uint32_t bpb, uint64_t* rows, double* coef, const uint32_t* kept,
                     unsigned long long* out_cursor, DevCounters* ctr, uint32_t cap, cudaStream_t s) {
        const unsigned blocks = (n_bins + bpb - 1) / bpb;
        if (write)
            k_pair_join<W, G, true><<<blocks, kThreads, 0, s>>>(rk, rc, start, n_bins, bpb, g, rows, coef, kept,
                                                                 out_cursor, ctr, cap);
        else
            k_pair_join<W, G, false><<<blocks, kThreads, 0, s>>>(rk, rc, start, n_bins, bpb, g, rows, coef, kept,
                                                                  out_cursor, ctr, cap);
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

template <int W>
void join2_launch(const PairDress& d, const uint64_t* rk, const double* rc, const uint32_t* start, uint32_t n_bins,
                  uint32_t bpb, const PairTwo& t, DevCounters* ctr, cudaStream_t s) {
    TwoParts<W> o;
    for (int j = 0; j < W; ++j) {  // device layout: x words, then z words
        o.mask.x[j] = t.mask[j];
        o.mask.z[j] = t.mask[W + j];
        o.aval.x[j] = t.aval[j];
        o.aval.z[j] = t.aval[W + j];
    }
    for (int k = 0; k < 2; ++k) {
        o.rows[k] = t.rows[k];
        o.coef[k] = t.coef[k];
        o.kept[k] = t.kept[k];
        o.cursor[k] = t.cursor[k];
    }
    const unsigned blocks = (n_bins + bpb - 1) / bpb;
    k_pair_join2<W, OneGen<W>><<<blocks, kThreads, 0, s>>>(rk, rc, start, n_bins, bpb,
                                                           OneGen<W>{make_gen<W>(d.pkey, d.cos_t, d.sin_t)}, o, ctr);
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

void launch_pair_hist(const PairDress& d, const uint64_t* rows, int64_t M, int log2_bins, uint32_t* counts,
                      uint32_t* tile_kept, DevCounters* ctr, cudaStream_t s, const uint8_t* live) {
    if (M <= 0) return;
    with_provider(d, [&](auto L, auto g) {
        decltype(L)::hist(g, rows, M, 64 - log2_bins, counts, tile_kept, ctr, live, s);
    });
    note_launch();
}

void launch_pair_split(const PairDress& d, bool compact, bool scatter, const uint64_t* rows, const double* coef,
                       int64_t M, int log2_bins, uint32_t* cursor, uint32_t cap, uint64_t* rk, double* rc,
                       const uint32_t* tile_off, uint64_t* rows_out, double* coef_out, DevCounters* ctr,
                       cudaStream_t s, const uint8_t* live) {
    if (M <= 0 || !(compact || scatter)) return;
    with_provider(d, [&](auto L, auto g) {
        decltype(L)::split(g, compact, scatter, rows, coef, M, 64 - log2_bins, cursor, cap, rk, rc, tile_off,
                           rows_out, coef_out, live, ctr, s);
    });
    note_launch();
}

void launch_pair_join(const PairDress& d, bool write, const uint64_t* rk, const double* rc, const uint32_t* start,
                      int log2_bins, uint32_t bins_per_block, uint64_t* rows, double* coef, const uint32_t* kept,
                      unsigned long long* out_cursor, DevCounters* ctr, cudaStream_t s, uint32_t cap) {
    const uint32_t n_bins = 1u << log2_bins;
    with_provider(d, [&](auto L, auto g) {
        decltype(L)::join(g, write, rk, rc, start, n_bins, bins_per_block, rows, coef, kept, out_cursor, ctr, cap, s);
    });
    note_launch();
}

void launch_pair_join2(const PairDress& d, const uint64_t* rk, const double* rc, const uint32_t* start,
                       int log2_bins, uint32_t bins_per_block, const PairTwo& t, DevCounters* ctr, cudaStream_t s) {
    const uint32_t n_bins = 1u << log2_bins;
    switch (d.Wd) {
        case 1: join2_launch<1>(d, rk, rc, start, n_bins, bins_per_block, t, ctr, s); break;
        case 2: join2_launch<2>(d, rk, rc, start, n_bins, bins_per_block, t, ctr, s); break;
        default: join2_launch<4>(d, rk, rc, start, n_bins, bins_per_block, t, ctr, s); break;
    }
    note_launch();
}

void launch_key_group(int Wd, const uint64_t* rows, const double* coef, int64_t n, int log2_bins, int phase,
                      uint32_t* counts, uint64_t* rk, double* rc, uint32_t* ri, uint32_t bins_per_block,
                      uint64_t* rows_out, double* c_out, unsigned long long* out_cursor, DevCounters* ctr,
                      cudaStream_t s) {
    if (n <= 0) return;
    const int shift = 64 - log2_bins;
    const uint32_t n_bins = 1u << log2_bins;
    auto run = [&](auto wtag) {
        constexpr int W = decltype(wtag)::value;
        if (phase == 0) {
            k_key_hist<W><<<grid_cap(n, 8), kThreads, 0, s>>>(rows, n, shift, counts + 1);
        } else if (phase == 1) {
            const unsigned blocks = (unsigned)((n + 4 * kThreads - 1) / (4 * kThreads));
            k_key_split<W><<<blocks, kThreads, 0, s>>>(rows, coef, n, shift, counts + 1, rk, rc, ri);
        } else {
            static std::atomic<unsigned long long> attr{0};
            if (first_on_device(&attr))
                cudaFuncSetAttribute(k_key_join<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kKeyJoinSmem);
            const unsigned blocks = (n_bins + bins_per_block - 1) / bins_per_block;
            k_key_join<W><<<blocks, kThreads, kKeyJoinSmem, s>>>(rk, rc, ri, counts, n_bins, bins_per_block, rows_out,
                                                                 c_out, out_cursor, ctr);
        }
    };
    switch (Wd) {
        case 1: run(std::integral_constant<int, 1>{}); break;
        case 2: run(std::integral_constant<int, 2>{}); break;
        default: run(std::integral_constant<int, 4>{}); break;
    }
    note_launch();
}

void launch_flag_tiles(const uint8_t* flags, int64_t n, uint32_t* tile_kept, cudaStream_t s) {
    if (n <= 0) return;
    k_flag_tiles<<<(unsigned)((n + kDressTile - 1) / kDressTile), kThreads, 0, s>>>(flags, n, tile_kept);
    note_launch();
}

}  // namespace iqcc
