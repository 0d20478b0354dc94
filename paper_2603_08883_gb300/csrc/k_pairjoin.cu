// Dressing by pair partition: the merge of Eq. 5 (App. D Eq. 18, "insert if
// unique, else add") without a resident index and without random DRAM access.
//
// A string T that anticommutes with P pairs with exactly one other string,
// its partner Q = T xor P (q -> q xor P is a bijection, and Q anticommutes
// with P as T does).  Both members of a pair have the same pair key: the
// member whose bit at P's lowest set bit is clear (exactly one member has
// that bit clear).  So a partition of the anticommuting rows by a hash of
// their pair key puts both members of every present pair in the same bin,
// and the merge becomes a local join.  The 2^L bins (the top L bits of the
// hash, about a thousand rows each) are reached in two passes, each with a
// fan-out small enough to rank rows in shared memory, so that no pass takes
// a position from a global atomic:
//
//   1. k_pair_hist   (or the A, B, C pass before the dress) one pass over the
//                    keys: per tile of kDressTile rows, the commuting rows it
//                    keeps and its anticommuting rows per level-1 partition
//                    (the top L1 <= 11 bits of the bin), one column of a
//                    partition-major count matrix; exclusive scans turn both
//                    into output offsets.
//   2. k_pair_split  one block per tile, into the other row buffer: the
//                    commuting rows to the tile's offset (ranked by ballots),
//                    the anticommuting rows with their coefficient and bin
//                    to their partition's offset for this tile (ranked by
//                    shared-memory counters).
//   3. k_pair_part2  one block per level-1 partition: a histogram of the
//                    remaining L - L1 bin bits, bin starts, and a copy of the
//                    partition's rows ordered by bin (shared-memory counters
//                    again).
//   4. k_pair_join   one block per group of consecutive bins: the group's
//                    rows are matched by pair key in a shared-memory table,
//                    each row is written behind the commuting rows with
//                    C_T cos(tau) - s_T C_Q sin(tau) (partner present, i T P =
//                    s_T Q) or C_T cos(tau) (partner absent), and each row
//                    without a partner appends (Q, s_T C_T sin(tau)).
//
// Every pass streams.  No per-generator index is built or maintained, so
// compressing H moves rows without any index upkeep.  The appended strings
// are absent from H by construction (a present partner would have been found
// in the same bin), so no duplicate merge is needed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "bulk.cuh"
#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;
constexpr int kJoinCap = 4096;             // rows one join block can hold
constexpr int kJoinSlots = 8192;           // its shared-memory table (load <= 1/2)
constexpr uint32_t kJoinEmpty = 0xFFFFFFFFu;
constexpr uint16_t kNoPartner = 0xFFFFu;
constexpr int kJoinTarget = 2048;          // rows per join block on average
constexpr int kPart2Threads = 512;

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

// Exclusive scan over the block of one value per thread (warp_tot: one entry
// per warp of the block).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* warp_tot) {
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

// Per tile of kDressTile rows: counts[d * n_tiles + tile] = its anticommuting
// rows in level-1 partition d (< 2^L1), tile_kept[tile] = its commuting live
// rows; the anticommuting total is added to ctr->n_anti.
template <int W, class G>
__global__ void __launch_bounds__(kThreads) k_pair_hist(const uint64_t* __restrict__ rows, int64_t M, G gen_of,
                                                        int L, uint32_t* counts, uint32_t* tile_kept,
                                                        DevCounters* ctr, const uint8_t* __restrict__ live) {
    __shared__ uint32_t s_h[1 << kPairL1Max];
    __shared__ uint32_t s_kept;
    const int L1 = pair_l1(L);
    const int F1 = 1 << L1;
    const int shift1 = 64 - L1;
    unsigned n_anti = 0;
    const int64_t n_tiles = (M + kDressTile - 1) / kDressTile;
    for (int d = threadIdx.x; d < F1; d += blockDim.x) s_h[d] = 0;
    if (threadIdx.x == 0) s_kept = 0;
    __syncthreads();
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        unsigned kept = 0;
        const int64_t end = min(M, (tile + 1) * kDressTile);
        for (int64_t i = tile * kDressTile + threadIdx.x; i < end; i += blockDim.x) {
            if (live && !live[i]) continue;
            const Key<W> t = load_key<W>(rows, i);
            const auto& g = gen_of(t);
            if (anticommutes<W>(t, g.p)) {
                atomicAdd(&s_h[pair_hash<W>(t, g.p, g.top_word, g.top_mask) >> shift1], 1u);
                ++n_anti;
            } else {
                ++kept;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kept += __shfl_down_sync(0xFFFFFFFFu, kept, o);
        if ((threadIdx.x & 31) == 0 && kept) atomicAdd(&s_kept, kept);
        __syncthreads();
        for (int d = threadIdx.x; d < F1; d += blockDim.x) {
            counts[(int64_t)d * n_tiles + tile] = s_h[d];
            s_h[d] = 0;
        }
        if (threadIdx.x == 0) {
            tile_kept[tile] = s_kept;
            s_kept = 0;
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_anti += __shfl_down_sync(0xFFFFFFFFu, n_anti, o);
    if ((threadIdx.x & 31) == 0 && n_anti) atomicAdd(&ctr->n_anti, (unsigned long long)n_anti);
}

// ---------------------------------------------------------------------------
// The split as a persistent kernel whose rows arrive by bulk copies.  Each
// block takes the tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... and walks
// them in chunks of 1024 rows; the chunks (keys, coefficients and, under a
// pending cut, live flags) are copied into a ring of kSplitStages shared-memory
// stages by cp.async.bulk with completion counted on one mbarrier per stage,
// kSplitStages - 1 chunks ahead of the one being worked on.  So the loads of
// later chunks are in flight while a chunk is ranked and written, which a
// one-shot tile (loads, then ranking, then stores) cannot do.  A partial chunk
// (the end of H) is read from global memory directly.  Every wait on an
// mbarrier is bounded by ctr->wait_limit polls; a wait that gives up records
// IQCC_ERR_TIMEOUT, waits (bounded again) for the copies still in flight, and
// the block returns.

// The level-1 copy of an anticommuting row is two whole-sector items: its key
// in k1 (stride pair_key_words(W), zero-padded to a sector) and a tail
// (coefficient, bin, 0, 0) in t1.  Written as whole sectors, no item is left
// partly written in L2 for another block to complete much later (which would
// make DRAM read the sector back first); the tails alone serve the second
// pass's histogram.
template <int W>
__device__ __forceinline__ void store_l1(uint64_t* k1, uint64_t* t1, uint32_t pos, const Key<W>& k, double c,
                                         uint32_t bin) {
    constexpr int KS = pair_key_words(W);
    uint64_t w[KS];
#pragma unroll
    for (int j = 0; j < W; ++j) {
        w[j] = k.x[j];
        w[W + j] = k.z[j];
    }
#pragma unroll
    for (int j = 2 * W; j < KS; ++j) w[j] = 0;
    uint64_t* p = k1 + (size_t)pos * KS;
#pragma unroll
    for (int j = 0; j < KS / 4; ++j) st256(p + 4 * j, w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
    st256(t1 + (size_t)pos * 4, (uint64_t)__double_as_longlong(c), bin, 0, 0);
}

template <int W>
__device__ __forceinline__ void load_l1(const uint64_t* k1, const uint64_t* t1, int64_t i, Key<W>& k, double& c,
                                        uint32_t& bin) {
    constexpr int KS = pair_key_words(W);
    uint64_t w[KS];
    const uint64_t* p = k1 + (size_t)i * KS;
#pragma unroll
    for (int j = 0; j < KS / 4; ++j) ld256(p + 4 * j, w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
#pragma unroll
    for (int j = 0; j < W; ++j) {
        k.x[j] = w[j];
        k.z[j] = w[W + j];
    }
    uint64_t a, b, u, v;
    ld256(t1 + (size_t)i * 4, a, b, u, v);
    c = __longlong_as_double((long long)a);
    bin = (uint32_t)b;
}

// A row's key as whole sectors to rows_out (16 W bytes, a multiple of 32 for W >= 2).
template <int W>
__device__ __forceinline__ void store_row(uint64_t* rows, int64_t i, const Key<W>& k) {
    if constexpr (W == 1) {
        store_key<W>(rows, i, k);
    } else {
        uint64_t w[2 * W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            w[j] = k.x[j];
            w[W + j] = k.z[j];
        }
        uint64_t* p = rows + (size_t)i * 2 * W;
#pragma unroll
        for (int j = 0; j < W / 2; ++j) st256(p + 4 * j, w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
    }
}

constexpr int kSplitChunk = 1024;
constexpr int kSplitStages = 2;
constexpr int kSplitChunks = kDressTile / kSplitChunk;

template <int W>
struct SplitStage {
    static constexpr size_t kKeys = (size_t)kSplitChunk * 16 * W;
    static constexpr size_t kCoefs = (size_t)kSplitChunk * 8;
    static constexpr size_t kLive = kSplitChunk;
    static constexpr size_t kBytes = kKeys + kCoefs + kLive;  // a multiple of 16
};

template <int W>
constexpr size_t split_smem_bytes() {
    return kSplitStages * SplitStage<W>::kBytes;
}

// Job j of a block: chunk j % kSplitChunks of its (j / kSplitChunks)-th tile.
// Thread 0 starts its copies into stage `st` (a full chunk), or, for a
// partial chunk or a job past the end, arrives on the stage's barrier without
// a copy.
template <int W>
__device__ __forceinline__ void split_issue(unsigned char* stage, uint64_t* bar, const uint64_t* rows,
                                            const double* coef, const uint8_t* live, int64_t n, int64_t r0) {
    if (r0 + kSplitChunk > n) {
        mbar_arrive(bar);
        return;
    }
    const uint32_t bytes =
        (uint32_t)(SplitStage<W>::kKeys + SplitStage<W>::kCoefs + (live ? SplitStage<W>::kLive : 0));
    fence_proxy_async_smem();
    mbar_expect_tx(bar, bytes);
    bulk_load(stage, rows + (size_t)r0 * 2 * W, (uint32_t)SplitStage<W>::kKeys, bar);
    bulk_load(stage + SplitStage<W>::kKeys, coef + r0, (uint32_t)SplitStage<W>::kCoefs, bar);
    if (live) bulk_load(stage + SplitStage<W>::kKeys + SplitStage<W>::kCoefs, live + r0, (uint32_t)SplitStage<W>::kLive, bar);
}

// The split, from the rows into the other row buffer: COMPACT copies the
// rows that commute with their generator to rows_out / coef_out from
// tile_off[t] on, in order (ranked by warp ballots); SCATTER copies each
// anticommuting row's key, coefficient and bin (the top L bits of its pair
// hash) to k1 / t1 (store_l1) at its level-1 partition's offset for the tile
// (base1: the exclusive scan of the counting pass's matrix), ranked by a
// shared-memory counter per partition.  No block waits on another and no
// position comes from a global atomic.  live (may be NULL): rows with
// live[i] == 0 (dropped by a pending term-limit cut) are neither kept nor
// copied.
template <int W, class G, bool COMPACT, bool SCATTER>
__global__ void __launch_bounds__(kThreads) k_pair_split(const uint64_t* __restrict__ rows,
                                                              const double* __restrict__ coef, int64_t n, G gen_of,
                                                              int L, const uint32_t* __restrict__ base1,
                                                              uint64_t* k1, uint64_t* t1,
                                                              const uint32_t* __restrict__ tile_off,
                                                              uint64_t* rows_out, double* coef_out,
                                                              const uint8_t* __restrict__ live, DevCounters* ctr) {
    extern __shared__ __align__(128) unsigned char s_stage[];
    __shared__ __align__(8) uint64_t s_bar[kSplitStages];
    __shared__ uint32_t s_cur[SCATTER ? (1 << kPairL1Max) : 1];
    __shared__ uint32_t s_w[kThreads / 32];
    constexpr int kPer = kSplitChunk / kThreads;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t n_tiles = (n + kDressTile - 1) / kDressTile;
    const int64_t my_tiles = n_tiles > (int64_t)blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t jobs = my_tiles * kSplitChunks;
    const int L1 = pair_l1(L);
    const int shift1 = 64 - L1, shiftL = 64 - L;
    const int limit = ctr->wait_limit;
    auto job_row = [&](int64_t j) {
        return ((int64_t)blockIdx.x + (j / kSplitChunks) * gridDim.x) * kDressTile + (j % kSplitChunks) * kSplitChunk;
    };
    if (threadIdx.x == 0) {
        for (int st = 0; st < kSplitStages; ++st) mbar_init(&s_bar[st], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int64_t j = 0; j < kSplitStages - 1 && j < jobs; ++j)
            split_issue<W>(s_stage + (size_t)j * SplitStage<W>::kBytes, &s_bar[j], rows, coef, live, n, job_row(j));
    uint32_t koff = 0;
    for (int64_t j = 0; j < jobs; ++j) {
        const int st = (int)(j % kSplitStages);
        const int64_t r0 = job_row(j);
        if (r0 >= n) break;  // the same for the whole block (only the last tile can end early)
        const int64_t t = r0 / kDressTile;
        if (threadIdx.x == 0 && j + kSplitStages - 1 < jobs) {
            const int64_t jn = j + kSplitStages - 1;
            const int sn = (int)(jn % kSplitStages);
            split_issue<W>(s_stage + (size_t)sn * SplitStage<W>::kBytes, &s_bar[sn], rows, coef, live, n,
                           job_row(jn));
        }
        if (j % kSplitChunks == 0) {  // a new tile: its offsets
            if (SCATTER)
                for (int d = threadIdx.x; d < (1 << L1); d += blockDim.x) s_cur[d] = base1[(int64_t)d * n_tiles + t];
            if (COMPACT) koff = tile_off[t];
            __syncthreads();
        }
        const bool ok = mbar_wait_bounded(&s_bar[st], (uint32_t)((j / kSplitStages) & 1), limit);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                set_error(ctr, IQCC_ERR_TIMEOUT, 75);
                // the copies still in flight land before the block's shared memory is released
                for (int64_t jj = j; jj < jobs && jj < j + kSplitStages; ++jj)
                    mbar_wait_bounded(&s_bar[jj % kSplitStages], (uint32_t)((jj / kSplitStages) & 1), limit);
            }
            return;
        }
        const unsigned char* stage = s_stage + (size_t)st * SplitStage<W>::kBytes;
        const bool full = r0 + kSplitChunk <= n;
        const double* s_coef = reinterpret_cast<const double*>(stage + SplitStage<W>::kKeys);
        const uint8_t* s_live = stage + SplitStage<W>::kKeys + SplitStage<W>::kCoefs;
        Key<W> key[kPer];
        double c[kPer];
        uint32_t pos[kPer], bin[kPer];
        bool keep[kPer], anti[kPer];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int rr = wid * (kPer * 32) + r * 32 + lane;
            const int64_t i = r0 + rr;
            keep[r] = anti[r] = false;
            bool in = i < n;
            if (in && live) in = full ? s_live[rr] != 0 : live[i] != 0;
            if (in) {
                if (full) {
                    key[r] = smem_key<W>(stage, rr);
                    c[r] = s_coef[rr];
                } else {
                    key[r] = load_key<W>(rows, i);
                    c[r] = coef[i];
                }
                const auto& g = gen_of(key[r]);
                anti[r] = anticommutes<W>(key[r], g.p);
                keep[r] = !anti[r];
                if (SCATTER && anti[r]) {
                    const uint64_t h = pair_hash<W>(key[r], g.p, g.top_word, g.top_mask);
                    pos[r] = atomicAdd(&s_cur[h >> shift1], 1u);
                    bin[r] = (uint32_t)(h >> shiftL);
                }
            }
        }
        if (SCATTER) {
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                if (anti[r]) {
                    store_l1<W>(k1, t1, pos[r], key[r], c[r], bin[r]);
                }
            }
        }
        if (COMPACT) {
            uint32_t rank[kPer];
            uint32_t wcount = 0;
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                const unsigned b = __ballot_sync(0xFFFFFFFFu, keep[r]);
                rank[r] = wcount + __popc(b & lt);
                wcount += __popc(b);
            }
            if (lane == 0) s_w[wid] = wcount;
            __syncthreads();
            uint32_t off = koff, tot = 0;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) {
                const uint32_t v = s_w[w];
                off += w < wid ? v : 0u;
                tot += v;
            }
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                if (keep[r]) {
                    store_row<W>(rows_out, (int64_t)(off + rank[r]), key[r]);
                    coef_out[off + rank[r]] = c[r];
                }
            }
            koff += tot;
        }
        __syncthreads();  // stage st and s_w are reused
    }
}

// The second level: block p orders level-1 partition p (items
// [base1[p * n_tiles], base1[(p + 1) * n_tiles]) of k1 / t1) by the low L2 =
// L - L1 bits of each record's bin into rk / rc, and writes the starts of its
// 2^L2 bins to start[(p << L2) ...] (the last block also start[2^L]).  Two
// reads of the bins (histogram, then placement through shared-memory
// counters) and one of the keys and coefficients.
template <int W>
__global__ void __launch_bounds__(kPart2Threads) k_pair_part2(int64_t n_tiles, int L,
                                                              const uint32_t* __restrict__ base1,
                                                              const uint64_t* __restrict__ k1,
                                                              const uint64_t* __restrict__ t1, uint64_t* rk,
                                                              double* rc, uint32_t* start) {
    constexpr int kU = 4;
    __shared__ uint32_t s_h[1 << kPairL2Max];
    __shared__ uint32_t s_warp[kPart2Threads / 32];
    const int L1 = pair_l1(L), L2 = L - L1;
    const uint32_t F2 = 1u << L2, mask = F2 - 1u;
    const int64_t p = blockIdx.x;
    const int64_t s = base1[p * n_tiles], e = base1[(p + 1) * n_tiles];
    for (uint32_t d = threadIdx.x; d < F2; d += blockDim.x) s_h[d] = 0;
    __syncthreads();
    for (int64_t i0 = s + threadIdx.x; i0 < e; i0 += (int64_t)blockDim.x * kU) {
        uint32_t b[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x;
            b[u] = i < e ? (uint32_t)__ldg(t1 + (size_t)i * 4 + 1) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + (int64_t)u * blockDim.x < e) atomicAdd(&s_h[b[u] & mask], 1u);
    }
    __syncthreads();
    // exclusive scan of the F2 counters: each thread takes a run of `per`
    const uint32_t per = (F2 + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(F2, threadIdx.x * per), hi = min(F2, lo + per);
    uint32_t run = 0;
    for (uint32_t d = lo; d < hi; ++d) run += s_h[d];
    uint32_t acc = block_excl_scan(run, s_warp);
    for (uint32_t d = lo; d < hi; ++d) {
        const uint32_t v = s_h[d];
        s_h[d] = acc;
        start[(p << L2) + d] = (uint32_t)s + acc;
        acc += v;
    }
    if (p == (int64_t)gridDim.x - 1 && threadIdx.x == 0) start[(int64_t)gridDim.x << L2] = (uint32_t)e;
    __syncthreads();
    for (int64_t i0 = s + threadIdx.x; i0 < e; i0 += (int64_t)blockDim.x * kU) {
        Key<W> key[kU];
        double c[kU];
        uint32_t b[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x;
            if (i < e) load_l1<W>(k1, t1, i, key[u], c[u], b[u]);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x;
            if (i < e) {
                const int64_t q = s + atomicAdd(&s_h[b[u] & mask], 1u);
                store_key<W>(rk, q, key[u]);
                rc[q] = c[u];
            }
        }
    }
}

// Block j joins bins [j*bpb, (j+1)*bpb): records [start[b0], start[b1]).
// WRITE: the dressed rows go to rows/coef from *kept on (the commuting rows
// end there), each block's at the position it reserves on out_cursor;
// appended partners follow the block's own rows.  Always: the number of rows
// without a partner is added to ctr->n_new.
template <int W, class G, bool WRITE>
__global__ void __launch_bounds__(kThreads) k_pair_join(const uint64_t* __restrict__ rk, const double* __restrict__ rc,
                                                        const uint32_t* __restrict__ start, uint32_t n_bins,
                                                        uint32_t bins_per_block, G gen_of, uint64_t* rows,
                                                        double* coef, const uint32_t* __restrict__ kept,
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
        if (WRITE) s_base = (unsigned long long)*kept + atomicAdd(out_cursor, (unsigned long long)(n + n_single));
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

// The launches for one provider type.
template <int W, class G>
struct PairLaunch {
    static void hist(const G& g, const uint64_t* rows, int64_t M, int L, uint32_t* counts, uint32_t* tile_kept,
                     DevCounters* ctr, const uint8_t* live, cudaStream_t s) {
        const int64_t n_tiles = (M + kDressTile - 1) / kDressTile;
        const int grid = (int)std::min<int64_t>(n_tiles, (int64_t)sm_count() * 4);
        k_pair_hist<W, G><<<grid, kThreads, 0, s>>>(rows, M, g, L, counts, tile_kept, ctr, live);
    }
    static void split(const G& g, bool compact, bool scatter, const uint64_t* rows, const double* coef, int64_t M,
                      int L, const uint32_t* base1, uint64_t* k1, uint64_t* t1,
                      const uint32_t* tile_off, uint64_t* rows_out, double* coef_out, const uint8_t* live,
                      DevCounters* ctr, cudaStream_t s) {
        const int64_t n_tiles = (M + kDressTile - 1) / kDressTile;
        constexpr size_t smem = split_smem_bytes<W>();
        const int per_sm = std::max(1, (int)((200 * 1024) / (smem + 9 * 1024)));
        const int grid = (int)std::min<int64_t>(n_tiles, (int64_t)sm_count() * per_sm);
        static std::atomic<unsigned long long> attr{0};
        if (first_on_device(&attr)) {
            cudaFuncSetAttribute(k_pair_split<W, G, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(k_pair_split<W, G, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(k_pair_split<W, G, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        }
        if (compact && scatter)
            k_pair_split<W, G, true, true><<<grid, kThreads, smem, s>>>(rows, coef, M, g, L, base1, k1, t1,
                                                                       tile_off, rows_out, coef_out, live, ctr);
        else if (compact)
            k_pair_split<W, G, true, false><<<grid, kThreads, smem, s>>>(rows, coef, M, g, L, base1, k1, t1,
                                                                        tile_off, rows_out, coef_out, live, ctr);
        else
            k_pair_split<W, G, false, true><<<grid, kThreads, smem, s>>>(rows, coef, M, g, L, base1, k1, t1,
                                                                        tile_off, rows_out, coef_out, live, ctr);
    }
    static void join(const G& g, bool write, const uint64_t* rk, const double* rc, const uint32_t* start,
                     uint32_t n_bins, uint32_t bpb, uint64_t* rows, double* coef, const uint32_t* kept,
                     unsigned long long* out_cursor, DevCounters* ctr, cudaStream_t s) {
        const unsigned blocks = (n_bins + bpb - 1) / bpb;
        if (write)
            k_pair_join<W, G, true><<<blocks, kThreads, 0, s>>>(rk, rc, start, n_bins, bpb, g, rows, coef, kept,
                                                                 out_cursor, ctr);
        else
            k_pair_join<W, G, false><<<blocks, kThreads, 0, s>>>(rk, rc, start, n_bins, bpb, g, rows, coef, kept,
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
// anticommuting), at least 1024 bins, at most 2^(kPairL1Max + kPairL2Max).
int pair_bins_log2(int64_t M) {
    int k = 10;
    while (k < kPairL1Max + kPairL2Max && ((int64_t)1 << k) * kJoinTarget < M) ++k;
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
        decltype(L)::hist(g, rows, M, log2_bins, counts, tile_kept, ctr, live, s);
    });
    note_launch();
}

void launch_pair_split(const PairDress& d, bool compact, bool scatter, const uint64_t* rows, const double* coef,
                       int64_t M, int log2_bins, const uint32_t* base1, uint64_t* k1, uint64_t* t1,
                       const uint32_t* tile_off, uint64_t* rows_out, double* coef_out, DevCounters* ctr,
                       cudaStream_t s, const uint8_t* live) {
    if (M <= 0 || !(compact || scatter)) return;
    with_provider(d, [&](auto L, auto g) {
        decltype(L)::split(g, compact, scatter, rows, coef, M, log2_bins, base1, k1, t1, tile_off, rows_out,
                           coef_out, live, ctr, s);
    });
    note_launch();
}

void launch_pair_part2(int Wd, int64_t M, int log2_bins, const uint32_t* base1, const uint64_t* k1,
                       const uint64_t* t1, uint64_t* rk, double* rc, uint32_t* start,
                       cudaStream_t s) {
    const int64_t n_tiles = (std::max<int64_t>(M, 1) + kDressTile - 1) / kDressTile;
    const unsigned parts = 1u << pair_l1(log2_bins);
    switch (Wd) {
        case 1: k_pair_part2<1><<<parts, kPart2Threads, 0, s>>>(n_tiles, log2_bins, base1, k1, t1, rk, rc, start); break;
        case 2: k_pair_part2<2><<<parts, kPart2Threads, 0, s>>>(n_tiles, log2_bins, base1, k1, t1, rk, rc, start); break;
        default: k_pair_part2<4><<<parts, kPart2Threads, 0, s>>>(n_tiles, log2_bins, base1, k1, t1, rk, rc, start); break;
    }
    note_launch();
}

void launch_pair_join(const PairDress& d, bool write, const uint64_t* rk, const double* rc, const uint32_t* start,
                      int log2_bins, uint32_t bins_per_block, uint64_t* rows, double* coef, const uint32_t* kept,
                      unsigned long long* out_cursor, DevCounters* ctr, cudaStream_t s) {
    const uint32_t n_bins = 1u << log2_bins;
    with_provider(d, [&](auto L, auto g) {
        decltype(L)::join(g, write, rk, rc, start, n_bins, bins_per_block, rows, coef, kept, out_cursor, ctr, s);
    });
    note_launch();
}

}  // namespace iqcc
