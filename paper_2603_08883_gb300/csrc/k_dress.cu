// The key index and the partitioned dressing (App. B's bit-wise partitions).
//
// Index: 2^k buckets of 4 eight-byte slots (one 32-byte sector), linear
// probing bucket by bucket; a slot holds an entry (fingerprint, distance from
// the home bucket, row; see make_entry) or kEmptySlot.  Lookups stop at the
// first empty slot.  A context builds it only for the partitioned dress, which
// looks its own rows up by key (the single-Hamiltonian and batched dresses
// join by pair partition instead, k_pairjoin.cu); any change of the rows
// invalidates it and the next partitioned dress rebuilds it (k_build.cu).
#include <cuda_runtime.h>

#include <atomic>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;

// Row index of key q, -1 when absent, -2 when the probe bound was reached.
// When absent, *free_slot is the empty slot that ended the probe: where q
// would be inserted.  Read-only use of the slots through the non-coherent
// path: a slot read stale can only be an empty slot since filled with a key
// that no lookup of the same pass seeks (an appended key is the partner of
// exactly one received row).
template <int W>
__device__ __forceinline__ int64_t lookup_slot(const Key<W>& q, uint64_t hv, const HashView& h,
                                               const uint64_t* __restrict__ rows, uint64_t* free_slot) {
    uint64_t b = hv & h.bucket_mask;
    for (int p = 0; p < h.max_probe; ++p) {
        const ulonglong2* s = reinterpret_cast<const ulonglong2*>(h.slots + b * kBucketSlots);
        const ulonglong2 s01 = __ldg(s), s23 = __ldg(s + 1);
        const uint64_t sl[4] = {s01.x, s01.y, s23.x, s23.y};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (sl[k] == kEmptySlot) {
                *free_slot = b * kBucketSlots + k;
                return -1;
            }
            if (fp_match(sl[k], hv)) {
                const uint32_t idx = (uint32_t)sl[k];
                const Key<W> r = load_key<W>(rows, idx);
                if (key_equal<W>(r, q)) return (int64_t)idx;
            }
        }
        b = (b + 1) & h.bucket_mask;
    }
    return -2;
}

// Insert the key with hash hv (proven absent) for `row` at `slot`, the empty
// slot its lookup ended on, or, if another insertion took that slot since, at
// the next empty slot of its probe sequence, within max_probe buckets of its
// home bucket.  The entry records its distance from home.
__device__ __forceinline__ bool insert_from(uint64_t hv, uint32_t row, uint64_t slot, const HashView& h) {
    unsigned long long* base = reinterpret_cast<unsigned long long*>(h.slots);
    const uint64_t b0 = hv & h.bucket_mask;
    uint64_t b = slot / kBucketSlots;
    int k0 = (int)(slot % kBucketSlots);
    for (int p = (int)((b - b0) & h.bucket_mask); p < h.max_probe; ++p) {
        const unsigned long long e = make_entry(hv, row, (uint64_t)p);
        for (int k = k0; k < 4; ++k) {
            unsigned long long* s = base + b * kBucketSlots + k;
            if (__ldcg(s) == kEmptySlot && atomicCAS(s, (unsigned long long)kEmptySlot, e) == kEmptySlot) return true;
        }
        k0 = 0;
        b = (b + 1) & h.bucket_mask;
    }
    return false;
}

__global__ void k_hash_clear(uint64_t* slots, uint64_t n) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    ulonglong2* p = reinterpret_cast<ulonglong2*>(slots);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n / 2; i += stride)
        p[i] = make_ulonglong2(kEmptySlot, kEmptySlot);
}

// Index rows [lo, hi) into a cleared table: one row per thread, occupied slots
// skipped by a plain read before the CAS.
template <int W>
__global__ void __launch_bounds__(kThreads) k_hash_insert(const uint64_t* __restrict__ rows, int64_t lo,
                                                          int64_t hi, HashView h, DevCounters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hi; i += stride) {
        const uint64_t hv = hash_key<W>(load_key<W>(rows, i));
        uint64_t b = hv & h.bucket_mask;
        bool done = false;
        for (int p = 0; p < h.max_probe && !done; ++p) {
            const unsigned long long entry = make_entry(hv, (uint32_t)i, (uint64_t)p);
            unsigned long long* s = reinterpret_cast<unsigned long long*>(h.slots + b * kBucketSlots);
            for (int k = 0; k < 4 && !done; ++k)
                done = s[k] == kEmptySlot && atomicCAS(s + k, (unsigned long long)kEmptySlot, entry) == kEmptySlot;
            b = (b + 1) & h.bucket_mask;
        }
        if (!done) set_error(ctr, IQCC_ERR_HASH_FULL, 1);
    }
}

// As lookup_slot, and loads the partner's coefficient together with its key
// (both depend only on the candidate row), so the caller needs no further
// dependent load for a found pair.
template <int W>
__device__ __forceinline__ int64_t lookup_slot_coef(const Key<W>& q, uint64_t hv, const HashView& h,
                                                    const uint64_t* __restrict__ rows, const double* coef,
                                                    uint64_t* free_slot, double* cq) {
    uint64_t b = hv & h.bucket_mask;
    for (int p = 0; p < h.max_probe; ++p) {
        const ulonglong2* s = reinterpret_cast<const ulonglong2*>(h.slots + b * kBucketSlots);
        const ulonglong2 s01 = __ldg(s), s23 = __ldg(s + 1);
        const uint64_t sl[4] = {s01.x, s01.y, s23.x, s23.y};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (sl[k] == kEmptySlot) {
                *free_slot = b * kBucketSlots + k;
                return -1;
            }
            if (fp_match(sl[k], hv)) {
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

// Partitioned dressing.  When H is split over several contexts by key bits
// and P flips one of those bits, the partner Q = T xor P of every
// anticommuting row T lies in the peer partition, so the pair rotation of
// Eq. 5 takes one exchange: each side sends its anticommuting rows to the
// peer (k_cross_rows), updates its own rows from the received ones
// (k_cross_local: C_K <- C_K cos + s_T C_T sin for the received T = K xor P,
// where i T P = s_T P(K)), and appends the partners that have no row on its
// side (k_cross_append: (K, s_T C_T sin)).

// The anticommuting rows, appended (warp-aggregated) as x [.][W], z [.][W], c.
template <int W>
__global__ void __launch_bounds__(kThreads) k_cross_rows(const uint64_t* __restrict__ rows,
                                                         const double* __restrict__ coef, int64_t M, Key<W> p,
                                                         int Wout, int64_t cap, uint64_t* ox, uint64_t* oz,
                                                         double* oc, unsigned long long* n_out) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t M32 = (M + 31) & ~(int64_t)31;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M32; i += stride) {
        Key<W> t{};
        bool a = false;
        if (i < M) {
            t = load_key<W>(rows, i);
            a = anticommutes<W>(t, p);
        }
        const unsigned m = __ballot_sync(FULL, a);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(n_out, (unsigned long long)__popc(m));
        base = __shfl_sync(FULL, base, leader);
        if (a) {
            const int64_t r = (int64_t)base + __popc(m & ((1u << lane) - 1u));
            if (r < cap) {
                for (int j = 0; j < Wout; ++j) {
                    ox[r * Wout + j] = t.x[j];
                    oz[r * Wout + j] = t.z[j];
                }
                oc[r] = coef[i];
            }
        }
    }
}

// Local rows: C_K <- C_K cos(tau) + s_T C_T sin(tau) when the peer holds
// T = K xor P (looked up in the peer's rows through their own index).
template <int W>
__global__ void __launch_bounds__(kThreads) k_cross_local(const uint64_t* __restrict__ rows, double* coef, int64_t M,
                                                          Gen<W> g, HashView hp, const uint64_t* __restrict__ prow,
                                                          const double* __restrict__ pcoef, DevCounters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        const Key<W> k = load_key<W>(rows, i);
        if (!anticommutes<W>(k, g.p)) continue;
        const Key<W> t = key_xor<W>(k, g.p);
        uint64_t fslot = 0;
        double ct = 0.0;
        const int64_t j = lookup_slot_coef<W>(t, hash_key<W>(t), hp, prow, pcoef, &fslot, &ct);
        const double ck = coef[i];
        if (j >= 0) {
            const double s = (double)product_sign<W>(t, g.yP, g.p, k);
            coef[i] = ck * g.cos_t + s * ct * g.sin_t;
        } else if (j == -1) {
            coef[i] = ck * g.cos_t;
        } else {
            set_error(ctr, IQCC_ERR_HASH_FULL, 60);
        }
    }
}

// Received rows T whose partner K = T xor P has no local row: append
// (K, s_T C_T sin(tau)) behind the M local rows and index it.
template <int W>
__global__ void __launch_bounds__(kThreads) k_cross_append(const uint64_t* __restrict__ prow,
                                                           const double* __restrict__ pcoef, int64_t n_peer, Gen<W> g,
                                                           const uint64_t* __restrict__ rows, uint64_t* rows_app,
                                                           double* coef, int64_t M, HashView h, DevCounters* ctr) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n32 = (n_peer + 31) & ~(int64_t)31;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n32; j += stride) {
        bool append = false;
        Key<W> k{};
        uint64_t hv = 0, fslot = 0;
        double c_new = 0.0;
        if (j < n_peer) {
            const Key<W> t = load_key<W>(prow, j);
            if (anticommutes<W>(t, g.p)) {
                k = key_xor<W>(t, g.p);
                hv = hash_key<W>(k);
                const int64_t idx = lookup_slot<W>(k, hv, h, rows, &fslot);
                if (idx == -1) {
                    append = true;
                    c_new = (double)product_sign<W>(t, g.yP, g.p, k) * pcoef[j] * g.sin_t;
                } else if (idx == -2) {
                    set_error(ctr, IQCC_ERR_HASH_FULL, 61);
                }
            }
        }
        const unsigned need = __ballot_sync(FULL, append);
        if (!need) continue;
        const int leader = __ffs(need) - 1;
        unsigned long long slot0 = 0;
        if (lane == leader) slot0 = atomicAdd(&ctr->n_new, (unsigned long long)__popc(need));
        slot0 = __shfl_sync(FULL, slot0, leader);
        if (append) {
            const int64_t r = M + (int64_t)slot0 + __popc(need & lt);
            store_key<W>(rows_app, r, k);
            coef[r] = c_new;
            if (!insert_from(hv, (uint32_t)r, fslot, h)) set_error(ctr, IQCC_ERR_HASH_FULL, 62);
        }
    }
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

void launch_cross_rows(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* pkey, int Wout,
                       int64_t cap, uint64_t* ox, uint64_t* oz, double* oc, unsigned long long* n_out,
                       cudaStream_t s) {
    if (M <= 0) return;
    const int grid = grid_for(M, 8);
    switch (Wd) {
        case 1: k_cross_rows<1><<<grid, kThreads, 0, s>>>(rows, coef, M, make_gen<1>(pkey, 1, 0).p, Wout, cap, ox, oz, oc, n_out); break;
        case 2: k_cross_rows<2><<<grid, kThreads, 0, s>>>(rows, coef, M, make_gen<2>(pkey, 1, 0).p, Wout, cap, ox, oz, oc, n_out); break;
        default: k_cross_rows<4><<<grid, kThreads, 0, s>>>(rows, coef, M, make_gen<4>(pkey, 1, 0).p, Wout, cap, ox, oz, oc, n_out); break;
    }
    note_launch();
}

void launch_cross_dress(int Wd, const uint64_t* rows, double* coef, int64_t M, const uint64_t* pkey, double cos_t,
                        double sin_t, HashView h, HashView hp, const uint64_t* prow, const double* pcoef,
                        int64_t n_peer, DevCounters* ctr, cudaStream_t s) {
    const int g1 = grid_for(M, 8), g2 = grid_for(n_peer, 8);
    uint64_t* rows_app = const_cast<uint64_t*>(rows);
    switch (Wd) {
        case 1: {
            const Gen<1> g = make_gen<1>(pkey, cos_t, sin_t);
            if (M > 0) k_cross_local<1><<<g1, kThreads, 0, s>>>(rows, coef, M, g, hp, prow, pcoef, ctr);
            if (n_peer > 0) k_cross_append<1><<<g2, kThreads, 0, s>>>(prow, pcoef, n_peer, g, rows, rows_app, coef, M, h, ctr);
            break;
        }
        case 2: {
            const Gen<2> g = make_gen<2>(pkey, cos_t, sin_t);
            if (M > 0) k_cross_local<2><<<g1, kThreads, 0, s>>>(rows, coef, M, g, hp, prow, pcoef, ctr);
            if (n_peer > 0) k_cross_append<2><<<g2, kThreads, 0, s>>>(prow, pcoef, n_peer, g, rows, rows_app, coef, M, h, ctr);
            break;
        }
        default: {
            const Gen<4> g = make_gen<4>(pkey, cos_t, sin_t);
            if (M > 0) k_cross_local<4><<<g1, kThreads, 0, s>>>(rows, coef, M, g, hp, prow, pcoef, ctr);
            if (n_peer > 0) k_cross_append<4><<<g2, kThreads, 0, s>>>(prow, pcoef, n_peer, g, rows, rows_app, coef, M, h, ctr);
            break;
        }
    }
    note_launch((M > 0) + (n_peer > 0));
}

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    return dev;
}

// Cached per device: a process may use several GPUs of different sizes.
int sm_count() {
    constexpr int kDevices = 64;
    static std::atomic<int> counts[kDevices];
    const int dev = current_device();
    int n = dev >= 0 && dev < kDevices ? counts[dev].load(std::memory_order_relaxed) : 0;
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        if (n <= 0) n = 1;
        if (dev >= 0 && dev < kDevices) counts[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

bool first_on_device(std::atomic<unsigned long long>* seen) {
    const int dev = current_device();
    if (dev < 0 || dev >= 64) return true;
    const unsigned long long bit = 1ull << dev;
    return (seen->fetch_or(bit, std::memory_order_relaxed) & bit) == 0;
}

int device_words(int n) { return n <= 64 ? 1 : (n <= 128 ? 2 : 4); }

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }

void launch_hash_clear(HashView h, uint64_t slots, cudaStream_t s) {
    k_hash_clear<<<grid_for_slots(slots), kThreads, 0, s>>>(h.slots, slots); note_launch();
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

}  // namespace iqcc
