// Dressing of the resident Hamiltonian by one generator (Eq. 5 in the
// library convention, Eq. 6) and the open-addressing index it relies on.
//
// Index: 2^k buckets of 4 eight-byte slots (one 32-byte sector); a slot holds
// (fingerprint32 << 32) | row32, kEmptySlot when never used and kTombSlot
// when its row was removed by compression.  Lookups skip tombstones and stop
// at the first empty slot.  Compression does not rebuild the index: it remaps
// every slot through the old-row -> new-row map of the compaction (removed
// rows become tombstones), and inserts reuse the first tombstone on a probe
// sequence, so tombstones are recycled by later dresses.
//
// Dress: one streaming pass over the M rows.  For a row T that anticommutes
// with P (popcount parity of (xT & zP) ^ (zT & xP)), its partner Q = T xor P is
// looked up.  Exactly one member of each present pair - the one with a zero at
// P's lowest set bit - rotates both coefficients; a row whose partner is
// absent scales itself by cos(tau) and appends (Q, s sin(tau) C_T) behind the
// M input rows, indexing it in the same pass.  q -> q xor P is a bijection, so
// appended keys are distinct and absent from H: no duplicate merge is needed
// within one generator (the "insert if unique, else add" merge of App. D,
// Eq. 18, done as a lookup).
#include <cuda_runtime.h>

#include <atomic>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ bool is_entry(uint64_t v) { return v != kEmptySlot && v != kTombSlot; }

// Row index of key q, -1 when absent, -2 when the probe bound was reached.
// When absent, *free_slot is the first tombstone met (else the empty slot that
// ended the probe) and *free_val its content: where q would be inserted.
// Read-only use of the slots through the non-coherent path: a slot read stale
// can only be empty or a tombstone that was since filled with a key that no
// lookup of this pass seeks (see k_dress).
template <int W>
__device__ __forceinline__ int64_t lookup_slot(const Key<W>& q, uint64_t hv, const HashView& h,
                                               const uint64_t* __restrict__ rows, uint64_t* free_slot,
                                               uint64_t* free_val) {
    const uint32_t fp = (uint32_t)(hv >> 32);
    uint64_t b = hv & h.bucket_mask;
    bool have_tomb = false;
    for (int p = 0; p < h.max_probe; ++p) {
        const ulonglong2* s = reinterpret_cast<const ulonglong2*>(h.slots + b * kBucketSlots);
        const ulonglong2 s01 = __ldg(s), s23 = __ldg(s + 1);
        const uint64_t sl[4] = {s01.x, s01.y, s23.x, s23.y};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (sl[k] == kEmptySlot) {
                if (!have_tomb) {
                    *free_slot = b * kBucketSlots + k;
                    *free_val = kEmptySlot;
                }
                return -1;
            }
            if (sl[k] == kTombSlot) {
                if (!have_tomb) {
                    have_tomb = true;
                    *free_slot = b * kBucketSlots + k;
                    *free_val = kTombSlot;
                }
                continue;
            }
            if ((uint32_t)(sl[k] >> 32) == fp) {
                const uint32_t idx = (uint32_t)sl[k];
                const Key<W> r = load_key<W>(rows, idx);
                if (key_equal<W>(r, q)) return (int64_t)idx;
            }
        }
        b = (b + 1) & h.bucket_mask;
    }
    return -2;
}

// Insert `entry` (a key proven absent) at `slot` if it still holds `expect`,
// else at the next empty or tombstone slot of its probe sequence.  *tomb tells
// whether the slot used held a tombstone.
__device__ __forceinline__ bool insert_from(uint64_t entry, uint64_t slot, uint64_t expect, const HashView& h,
                                            bool* tomb) {
    unsigned long long* base = reinterpret_cast<unsigned long long*>(h.slots);
    if (atomicCAS(base + slot, (unsigned long long)expect, (unsigned long long)entry) == expect) {
        *tomb = expect == kTombSlot;
        return true;
    }
    uint64_t b = slot / kBucketSlots;
    int k0 = (int)(slot % kBucketSlots) + 1;
    for (int p = 0; p < h.max_probe; ++p) {
        for (int k = k0; k < 4; ++k) {
            unsigned long long* s = base + b * kBucketSlots + k;
            unsigned long long v = __ldcg(s);
            while (!is_entry(v)) {
                const unsigned long long prev = atomicCAS(s, v, (unsigned long long)entry);
                if (prev == v) {
                    *tomb = v == kTombSlot;
                    return true;
                }
                v = prev;
            }
        }
        k0 = 0;
        b = (b + 1) & h.bucket_mask;
    }
    return false;
}

template <int W>
__device__ __forceinline__ bool bit_of(const Key<W>& k, int word, uint64_t mask) {
    uint64_t v = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        if (word == j) v = k.x[j];
        if (word == W + j) v = k.z[j];
    }
    return (v & mask) != 0;
}

__global__ void k_hash_clear(uint64_t* slots, uint64_t n) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    ulonglong2* p = reinterpret_cast<ulonglong2*>(slots);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n / 2; i += stride)
        p[i] = make_ulonglong2(kEmptySlot, kEmptySlot);
}

// Index rows [lo, hi) into a table without tombstones (a fresh build): one row
// per thread, occupied slots skipped by a plain read before the CAS.
template <int W>
__global__ void __launch_bounds__(kThreads) k_hash_insert(const uint64_t* __restrict__ rows, int64_t lo,
                                                          int64_t hi, HashView h, DevCounters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hi; i += stride) {
        const uint64_t hv = hash_key<W>(load_key<W>(rows, i));
        const uint64_t entry = (hv & 0xFFFFFFFF00000000ull) | (uint64_t)i;
        uint64_t b = hv & h.bucket_mask;
        bool done = false;
        for (int p = 0; p < h.max_probe && !done; ++p) {
            unsigned long long* s = reinterpret_cast<unsigned long long*>(h.slots + b * kBucketSlots);
            for (int k = 0; k < 4 && !done; ++k)
                done = s[k] == kEmptySlot &&
                       atomicCAS(s + k, (unsigned long long)kEmptySlot, (unsigned long long)entry) == kEmptySlot;
            b = (b + 1) & h.bucket_mask;
        }
        if (!done) set_error(ctr, IQCC_ERR_HASH_FULL, 1);
    }
}

// After an in-place compaction: entries of kept rows get their new row index,
// entries of removed rows become tombstones (new_row == kRowRemoved).
__global__ void k_hash_remap(uint64_t* slots, uint64_t n, const uint32_t* __restrict__ new_row) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    ulonglong2* p = reinterpret_cast<ulonglong2*>(slots);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n / 2; i += stride) {
        const ulonglong2 v = p[i];
        uint64_t w[2] = {v.x, v.y};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!is_entry(w[k])) continue;
            const uint32_t nr = __ldg(new_row + (uint32_t)w[k]);
            w[k] = (nr == kRowRemoved) ? kTombSlot : ((w[k] & 0xFFFFFFFF00000000ull) | (uint64_t)nr);
        }
        p[i] = make_ulonglong2(w[0], w[1]);
    }
}

// As lookup_slot, and loads the partner's coefficient together with its key
// (both depend only on the candidate row), so the caller needs no further
// dependent load for a found pair.
template <int W>
__device__ __forceinline__ int64_t lookup_slot_coef(const Key<W>& q, uint64_t hv, const HashView& h,
                                                    const uint64_t* __restrict__ rows, const double* coef,
                                                    uint64_t* free_slot, uint64_t* free_val, double* cq) {
    const uint32_t fp = (uint32_t)(hv >> 32);
    uint64_t b = hv & h.bucket_mask;
    bool have_tomb = false;
    for (int p = 0; p < h.max_probe; ++p) {
        const ulonglong2* s = reinterpret_cast<const ulonglong2*>(h.slots + b * kBucketSlots);
        const ulonglong2 s01 = __ldg(s), s23 = __ldg(s + 1);
        const uint64_t sl[4] = {s01.x, s01.y, s23.x, s23.y};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (sl[k] == kEmptySlot) {
                if (!have_tomb) {
                    *free_slot = b * kBucketSlots + k;
                    *free_val = kEmptySlot;
                }
                return -1;
            }
            if (sl[k] == kTombSlot) {
                if (!have_tomb) {
                    have_tomb = true;
                    *free_slot = b * kBucketSlots + k;
                    *free_val = kTombSlot;
                }
                continue;
            }
            if ((uint32_t)(sl[k] >> 32) == fp) {
                const uint32_t idx = (uint32_t)sl[k];
                const double c = coef[idx];
                const Key<W> r = load_key<W>(rows, idx);
                if (key_equal<W>(r, q)) {
                    *cq = c;
                    return (int64_t)idx;
                }
            }
        }
        b = (b + 1) & h.bucket_mask;
    }
    return -2;
}

constexpr int kWarpTile = 64;  // rows classified per warp before the probes
#ifndef IQCC_DRESS_MIN_BLOCKS
#define IQCC_DRESS_MIN_BLOCKS 4     // resident 256-thread blocks per SM the register budget targets (5 spills)
#endif

// One pass of Eq. 5 over rows [0, M).  Each warp classifies a tile of 64 rows
// (two per lane) and queues the anticommuting ones in shared memory, so that
// every lane then works on one queued row: partner lookup, pair rotation or
// append.  An appended partner is inserted into the index at the first free
// slot (tombstone or empty) its lookup met.  Concurrent inserts leave every
// lookup correct: a key present before the pass has no empty slot ahead of it
// in its probe sequence, and a slot filled during the pass only ever held an
// empty or a tombstone (which a lookup passes over or stops at) and receives a
// key no lookup seeks (an appended key is the partner of exactly one row,
// q -> q xor P being a bijection).  rows_app is the same buffer as rows;
// appended rows land at M + slot and are not visited by this pass.
template <int W>
__global__ void __launch_bounds__(kThreads, W == 4 ? 4 : IQCC_DRESS_MIN_BLOCKS) k_dress(const uint64_t* __restrict__ rows,
                                                                    uint64_t* rows_app, double* coef, int64_t M,
                                                                    Gen<W> g, HashView h, DevCounters* ctr) {
    __shared__ uint32_t s_queue[kThreads / 32][kWarpTile];
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t* queue = s_queue[wid];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned n_anti = 0;
    for (int64_t base = warp * kWarpTile; base < M; base += n_warps * kWarpTile) {
        int nq = 0;
#pragma unroll
        for (int r = 0; r < kWarpTile / 32; ++r) {
            const int64_t i = base + r * 32 + lane;
            bool a = false;
            if (i < M) a = anticommutes<W>(load_key<W>(rows, i), g.p);
            const unsigned m = __ballot_sync(FULL, a);
            if (a) queue[nq + __popc(m & lt)] = (uint32_t)(r * 32 + lane);
            nq += __popc(m);
        }
        __syncwarp();
        n_anti += (lane == 0) ? (unsigned)nq : 0u;
        for (int e0 = 0; e0 < nq; e0 += 32) {
            const int e = e0 + lane;
            bool append = false;
            Key<W> q;
            double c_new = 0.0;
            uint64_t hv = 0, fslot = 0, fval = kEmptySlot;
            if (e < nq) {
                const int64_t i = base + queue[e];
                const double ct = coef[i];  // independent of the lookup: issued first
                const Key<W> t = load_key<W>(rows, i);
                q = key_xor<W>(t, g.p);
                const double s = (double)product_sign<W>(t, g.yP, g.p, q);
                const bool upper = bit_of<W>(t, g.top_word, g.top_mask);
                hv = hash_key<W>(q);
                double cq = 0.0;
                const int64_t j = lookup_slot_coef<W>(q, hv, h, rows, coef, &fslot, &fval, &cq);
                if (j == -1) {
                    coef[i] = ct * g.cos_t;
                    c_new = s * ct * g.sin_t;
                    append = true;
                } else if (j >= 0) {
                    if (!upper) {
                        coef[i] = ct * g.cos_t - s * cq * g.sin_t;
                        coef[j] = cq * g.cos_t + s * ct * g.sin_t;
                    }
                } else {
                    set_error(ctr, IQCC_ERR_HASH_FULL, 2);
                }
            }
            const unsigned need = __ballot_sync(FULL, append);
            if (need) {
                const int leader = __ffs(need) - 1;
                unsigned long long slot0 = 0;
                if (lane == leader) slot0 = atomicAdd(&ctr->n_new, (unsigned long long)__popc(need));
                slot0 = __shfl_sync(FULL, slot0, leader);
                if (append) {
                    const int64_t r = M + (int64_t)slot0 + __popc(need & lt);
                    store_key<W>(rows_app, r, q);
                    coef[r] = c_new;
                    const uint64_t entry = (hv & 0xFFFFFFFF00000000ull) | (uint64_t)r;
                    bool tomb = false;
                    if (!insert_from(entry, fslot, fval, h, &tomb)) set_error(ctr, IQCC_ERR_HASH_FULL, 4);
                    else if (tomb) atomicAdd(&ctr->tomb_reused, 1ull);
                }
            }
        }
        __syncwarp();
    }
    if (lane == 0 && n_anti) atomicAdd(&ctr->n_anti, (unsigned long long)n_anti);
}

// Admission count: how many partners a dress would append (no writes to H).
template <int W>
__global__ void __launch_bounds__(kThreads) k_dress_count(const uint64_t* __restrict__ rows, int64_t M,
                                                          Gen<W> g, HashView h, DevCounters* ctr) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    unsigned cnt = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        Key<W> t = load_key<W>(rows, i);
        if (anticommutes<W>(t, g.p)) {
            Key<W> q = key_xor<W>(t, g.p);
            uint64_t fslot, fval;
            int64_t j = lookup_slot<W>(q, hash_key<W>(q), h, rows, &fslot, &fval);
            if (j == -1) ++cnt;
            else if (j == -2) set_error(ctr, IQCC_ERR_HASH_FULL, 3);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(FULL, cnt, o);
    if (lane == 0 && cnt) atomicAdd(&ctr->n_new, (unsigned long long)cnt);
}

template <int W>
Gen<W> make_gen(const uint64_t* pkey, double cos_t, double sin_t) {
    Gen<W> g{};
    int y = 0;
    g.top_word = -1;
    for (int j = 0; j < W; ++j) {
        g.p.x[j] = pkey[j];
        g.p.z[j] = pkey[W + j];
        y += __builtin_popcountll(pkey[j] & pkey[W + j]);
    }
    for (int w = 0; w < 2 * W && g.top_word < 0; ++w)
        if (pkey[w]) { g.top_word = w; g.top_mask = pkey[w] & (~pkey[w] + 1); }
    if (g.top_word < 0) { g.top_word = 0; g.top_mask = 0; }
    g.yP = y & 3;
    g.cos_t = cos_t;
    g.sin_t = sin_t;
    return g;
}

int grid_for(int64_t n, int per_sm) {
    int64_t want = (n + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)sm_count() * per_sm;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

int grid_for_slots(uint64_t slots) {
    int grid = (int)((slots / 2 + kThreads - 1) / kThreads);
    int cap = sm_count() * 8;
    if (grid > cap) grid = cap;
    return grid < 1 ? 1 : grid;
}

}  // namespace

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

int device_words(int n) { return n <= 64 ? 1 : (n <= 128 ? 2 : 4); }

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }

void launch_hash_clear(HashView h, uint64_t slots, cudaStream_t s) {
    k_hash_clear<<<grid_for_slots(slots), kThreads, 0, s>>>(h.slots, slots); note_launch();
}

void launch_hash_remap(HashView h, uint64_t slots, const uint32_t* new_row, cudaStream_t s) {
    k_hash_remap<<<grid_for_slots(slots), kThreads, 0, s>>>(h.slots, slots, new_row); note_launch();
}

void launch_hash_insert(int Wd, const uint64_t* rows, int64_t lo, int64_t hi, HashView h,
                        DevCounters* ctr, cudaStream_t s) {
    if (hi <= lo) return;
    int grid = grid_for(hi - lo, 8);
    switch (Wd) {
        case 1: k_hash_insert<1><<<grid, kThreads, 0, s>>>(rows, lo, hi, h, ctr); note_launch(); break;
        case 2: k_hash_insert<2><<<grid, kThreads, 0, s>>>(rows, lo, hi, h, ctr); note_launch(); break;
        default: k_hash_insert<4><<<grid, kThreads, 0, s>>>(rows, lo, hi, h, ctr); note_launch(); break;
    }
}

void launch_dress(int Wd, const uint64_t* rows_in, uint64_t* rows, double* coef, int64_t M,
                  const uint64_t* pkey, double cos_t, double sin_t, HashView h, DevCounters* ctr,
                  cudaStream_t s) {
    if (M <= 0) return;
    int grid = grid_for(M, 8);
    switch (Wd) {
        case 1: k_dress<1><<<grid, kThreads, 0, s>>>(rows_in, rows, coef, M, make_gen<1>(pkey, cos_t, sin_t), h, ctr); note_launch(); break;
        case 2: k_dress<2><<<grid, kThreads, 0, s>>>(rows_in, rows, coef, M, make_gen<2>(pkey, cos_t, sin_t), h, ctr); note_launch(); break;
        default: k_dress<4><<<grid, kThreads, 0, s>>>(rows_in, rows, coef, M, make_gen<4>(pkey, cos_t, sin_t), h, ctr); note_launch(); break;
    }
}

void launch_dress_count(int Wd, const uint64_t* rows, int64_t M, const uint64_t* pkey, HashView h,
                        DevCounters* ctr, cudaStream_t s) {
    if (M <= 0) return;
    int grid = grid_for(M, 8);
    switch (Wd) {
        case 1: k_dress_count<1><<<grid, kThreads, 0, s>>>(rows, M, make_gen<1>(pkey, 1, 0), h, ctr); note_launch(); break;
        case 2: k_dress_count<2><<<grid, kThreads, 0, s>>>(rows, M, make_gen<2>(pkey, 1, 0), h, ctr); note_launch(); break;
        default: k_dress_count<4><<<grid, kThreads, 0, s>>>(rows, M, make_gen<4>(pkey, 1, 0), h, ctr); note_launch(); break;
    }
}

}  // namespace iqcc
