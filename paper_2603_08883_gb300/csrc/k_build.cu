// Construction of the key index without global atomics on the table.
//
// The index (see k_dress.cu) is split into partitions of 8192 consecutive
// slots (64 KB).  A build hashes every row, orders the (hash, row) records by
// partition with stable 8-bit radix passes that stage each tile in shared
// memory (so the writes go out in runs), and then gives each partition to one
// block, which inserts its records into a copy of the partition held in shared
// memory by linear probing and writes the whole partition, empty slots
// included, in one coalesced sweep.  A record whose probe runs past the end of
// its partition is set aside and inserted afterwards, with global CAS, into
// the already written slots that follow, exactly as linear probing would have
// placed it.  The result is the same kind of table the dress kernel reads:
// every key sits at the first free slot of its probe sequence at the time it
// was placed, with no empty slot between its home bucket and its slot.
#include <cuda_runtime.h>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // records per block in a partition pass
constexpr int kDigitBits = 8;
constexpr int kBins = 1 << kDigitBits;
constexpr int kPartLog2 = 13;             // slots per partition: 8192 = 64 KB of shared memory

__device__ __forceinline__ uint32_t part_of(uint64_t h, uint64_t bucket_mask, int part_shift) {
    return (uint32_t)(((h & bucket_mask) * kBucketSlots) >> part_shift);
}

template <int W>
__global__ void k_build_hash(const uint64_t* __restrict__ rows, int64_t n, uint64_t* hrec) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s)
        hrec[i] = hash_key<W>(load_key<W>(rows, i));
}

// Per-block histograms of one digit of the partition index: hist[d * nblocks + block].
__global__ void k_part_hist(const uint64_t* __restrict__ h, int64_t n, uint64_t bmask, int pshift, int dshift,
                            uint32_t* hist, int64_t nblocks) {
    __shared__ uint32_t sh[kBins];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kItems; ++r) {
        const int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&sh[(part_of(h[i], bmask, pshift) >> dshift) & (kBins - 1)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = sh[threadIdx.x];
}

// Exclusive scan over the block of one value per thread (warp_tot: one entry per warp).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot) {
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

// One stable pass.  Each warp ranks its own contiguous 256 records (8 rounds
// of 32; lanes with the same digit find each other with match_any and the
// lowest of them advances the warp's counter for that digit), so no block-wide
// barrier is needed until the counts of all warps are combined.  Records are
// then staged in shared memory in digit order and written out in runs.
constexpr int kSThreads = 512;                // scatter block: 16 warps of 8 x 32 records
constexpr int kSItems = kTile / kSThreads;
constexpr int kSWarps = kSThreads / 32;

__global__ void __launch_bounds__(kSThreads, 2) k_part_scatter(const uint64_t* __restrict__ h_in,
                                                               const uint32_t* __restrict__ r_in, int64_t n,
                                                               uint64_t bmask, int pshift, int dshift,
                                                               const uint32_t* __restrict__ offsets, int64_t nblocks,
                                                               uint64_t* h_out, uint32_t* r_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* st_h = reinterpret_cast<uint64_t*>(smem_raw);
    uint32_t* st_r = reinterpret_cast<uint32_t*>(st_h + kTile);
    __shared__ uint32_t s_wh[kSWarps][kBins];  // per-warp digit counts, then per-warp offsets
    __shared__ uint32_t s_tile_off[kBins], s_glob[kBins], s_warp[kSWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kTile;
    const int64_t wbase = base + (int64_t)wid * (kSItems * 32);
    for (int d = lane; d < kBins; d += 32) s_wh[wid][d] = 0;
    __syncwarp();
    uint64_t hv[kSItems];
    uint32_t rv[kSItems];
    uint32_t pk[kSItems];  // digit << 16 | position among the warp's records of that digit
#pragma unroll
    for (int r = 0; r < kSItems; ++r) {
        const int64_t i = wbase + (int64_t)r * 32 + lane;
        uint32_t d = kBins;  // sentinel for the ragged tail
        hv[r] = 0;
        rv[r] = 0;
        if (i < n) {
            hv[r] = h_in[i];
            rv[r] = r_in ? r_in[i] : (uint32_t)i;
            d = (part_of(hv[r], bmask, pshift) >> dshift) & (kBins - 1);
        }
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
    // thread t < 256 owns digit t: offsets of each warp within the digit, then of the digit within the tile
    uint32_t tot = 0;
    if (threadIdx.x < kBins) {
        for (int w = 0; w < kSWarps; ++w) {
            const uint32_t c = s_wh[w][threadIdx.x];
            s_wh[w][threadIdx.x] = tot;
            tot += c;
        }
    }
    const uint32_t excl = block_exclusive_scan(tot, s_warp);
    if (threadIdx.x < kBins) {
        s_tile_off[threadIdx.x] = excl;
        s_glob[threadIdx.x] = offsets[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSItems; ++r) {
        const uint32_t d = pk[r] >> 16;
        if (d < kBins) {
            const uint32_t pos = s_tile_off[d] + s_wh[wid][d] + (pk[r] & 0xFFFFu);
            st_h[pos] = hv[r];
            st_r[pos] = rv[r];
        }
    }
    __syncthreads();
    const int64_t cnt = min((int64_t)kTile, n - base);
    for (int k = threadIdx.x; k < cnt; k += kSThreads) {
        const uint64_t hk = st_h[k];
        const uint32_t d = (part_of(hk, bmask, pshift) >> dshift) & (kBins - 1);
        const int64_t out = (int64_t)s_glob[d] + (k - (int64_t)s_tile_off[d]);
        h_out[out] = hk;
        r_out[out] = st_r[k];
    }
}

// start[p] = first record of partition p in the ordered records (start[P] = n).
__global__ void k_part_starts(const uint64_t* __restrict__ h, int64_t n, uint64_t bmask, int pshift, uint32_t P,
                              uint32_t* start) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += s) {
        const uint32_t cur = k < n ? part_of(h[k], bmask, pshift) : P;
        const uint32_t prev = k > 0 ? part_of(h[k - 1], bmask, pshift) : 0;
        const uint32_t lo = k > 0 ? prev + 1 : 0;
        for (uint32_t p = lo; p <= cur && p <= P; ++p) start[p] = (uint32_t)k;
    }
}

// Linear probing in a shared-memory copy of one partition, from the slot
// `home` (partition-relative, bucket-aligned) to the partition end and within
// max_slots of home.  Returns 1 when placed, 0 when the probe ran past the
// partition end, -1 when it reached the probe bound inside the partition.
__device__ __forceinline__ int place_local(unsigned long long* tab, uint32_t part_slots, uint32_t home,
                                           uint64_t hv_fp, uint32_t row, int max_slots) {
    for (uint32_t j = home; j < part_slots; ++j) {
        if ((int)(j - home) >= max_slots) return -1;
        if (tab[j] == kEmptySlot) {
            const unsigned long long e = make_entry(hv_fp, row, (uint64_t)((j - home) / kBucketSlots));
            if (atomicCAS(tab + j, (unsigned long long)kEmptySlot, e) == kEmptySlot) return 1;
        }
    }
    return 0;
}

__device__ __forceinline__ void list_overflow(uint64_t hv_fp, uint32_t row, uint64_t home_slot, uint64_t* ovf_entry,
                                              uint64_t* ovf_home, unsigned long long* n_ovf, int64_t ovf_cap,
                                              DevCounters* ctr, int where) {
    const unsigned long long at = atomicAdd(n_ovf, 1ull);
    if ((int64_t)at < ovf_cap) {
        ovf_entry[at] = make_entry(hv_fp, row, 0);
        ovf_home[at] = home_slot;
    } else {
        set_error(ctr, IQCC_ERR_HASH_FULL, where);
    }
}

// One block per partition: the partition's records are placed by linear
// probing in a shared-memory copy, which is then written out whole (empty
// slots included) in one coalesced sweep.  A record whose probe runs past the
// partition end is listed with its home slot.
__global__ void __launch_bounds__(kThreads) k_part_build(const uint64_t* __restrict__ h, const uint32_t* __restrict__ r,
                                                         const uint32_t* __restrict__ start, uint64_t bmask,
                                                         int pshift, int max_slots, uint64_t* slots,
                                                         uint64_t* ovf_entry, uint64_t* ovf_home,
                                                         unsigned long long* n_ovf, int64_t ovf_cap,
                                                         DevCounters* ctr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* tab = reinterpret_cast<unsigned long long*>(smem_raw);
    const uint32_t part_slots = 1u << pshift;
    for (uint32_t k = threadIdx.x; k < part_slots; k += blockDim.x) tab[k] = kEmptySlot;
    __syncthreads();
    const uint64_t first = (uint64_t)blockIdx.x << pshift;
    const uint32_t k0 = start[blockIdx.x], k1 = start[blockIdx.x + 1];
    for (uint32_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const uint64_t hv = h[k];
        const uint32_t home = (uint32_t)((hv & bmask) * kBucketSlots - first);
        const int res = place_local(tab, part_slots, home, hv, r[k], max_slots);
        if (res < 0) set_error(ctr, IQCC_ERR_HASH_FULL, 40);
        else if (res == 0) list_overflow(hv, r[k], first + home, ovf_entry, ovf_home, n_ovf, ovf_cap, ctr, 41);
    }
    __syncthreads();
    ulonglong2* out = reinterpret_cast<ulonglong2*>(slots + first);
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(tab);
    for (uint32_t k = threadIdx.x; k < part_slots / 2; k += blockDim.x) out[k] = src[k];
}

// The listed entries, inserted into the written table by global CAS: linear
// probing from the home slot (wrapping at the table end), within the probe
// bound, the stored distance set to the slot found.
__global__ void k_part_overflow(const uint64_t* __restrict__ ovf_entry, const uint64_t* __restrict__ ovf_home,
                                const unsigned long long* n_ovf, int64_t ovf_cap, uint64_t* slots,
                                uint64_t n_slots, int max_slots, DevCounters* ctr) {
    const int64_t n = min((int64_t)*n_ovf, ovf_cap);
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += s) {
        const uint64_t home = ovf_home[i];
        const uint64_t e0 = ovf_entry[i];
        bool done = false;
        for (int d = 0; d < max_slots && !done; ++d) {
            unsigned long long* sl = reinterpret_cast<unsigned long long*>(slots + ((home + d) & (n_slots - 1)));
            if (*sl != kEmptySlot) continue;
            const unsigned long long e = make_entry(e0, (uint32_t)e0, (uint64_t)(d / kBucketSlots));
            done = atomicCAS(sl, (unsigned long long)kEmptySlot, e) == kEmptySlot;
        }
        if (!done) set_error(ctr, IQCC_ERR_HASH_FULL, 42);
    }
}

// Exclusive scan of a long u32 array in three steps: chunk sums, a one-block
// scan of the sums, and a scan of each chunk from its offset.
constexpr int kScanChunkAlign = 1024;

__global__ void __launch_bounds__(kThreads) k_chunk_sums(const uint32_t* __restrict__ d, int64_t n, int64_t chunk,
                                                         uint32_t* sums) {
    __shared__ uint32_t sw[kThreads / 32];
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(n, lo + chunk);
    uint32_t s = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) s += d[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += sw[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void k_scan_small(uint32_t* v, int n) {  // n <= 1024, one block of 1024
    __shared__ uint32_t sh[1024];
    const int t = threadIdx.x;
    sh[t] = t < n ? v[t] : 0u;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t y = t >= off ? sh[t - off] : 0u;
        __syncthreads();
        sh[t] += y;
        __syncthreads();
    }
    if (t < n) v[t] = t ? sh[t - 1] : 0u;
}

__global__ void __launch_bounds__(kThreads) k_chunk_scan(uint32_t* d, int64_t n, int64_t chunk,
                                                         const uint32_t* __restrict__ offs) {
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ uint32_t s_tot;
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(n, lo + chunk);
    uint32_t run = offs[blockIdx.x];
    for (int64_t t0 = lo; t0 < hi; t0 += kThreads * 4) {
        const int64_t i = t0 + (int64_t)threadIdx.x * 4;
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (i + k < hi) ? d[i + k] : 0u;
        const uint32_t mine = v[0] + v[1] + v[2] + v[3];
        const uint32_t ex = block_exclusive_scan(mine, s_warp);
        if (threadIdx.x == kThreads - 1) s_tot = ex + mine;
        uint32_t acc = run + ex;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i + k < hi) d[i + k] = acc;
            acc += v[k];
        }
        __syncthreads();
        run += s_tot;
        __syncthreads();
    }
}

int grid_stride_blocks(int64_t n) {
    int64_t want = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

struct BuildPlan {
    int pshift;        // log2(slots per partition)
    uint32_t parts;    // partitions
    int pbits;         // log2(parts)
    int64_t nblocks;   // tiles of a partition pass
    int64_t ovf_cap;   // records that may probe past their partition
    int64_t scan_n;    // histogram length
    int scan_chunks;
    int64_t scan_chunk;
};

BuildPlan plan_for(int64_t n, uint64_t n_slots) {
    BuildPlan b;
    int slot_log2 = 0;
    while ((1ull << slot_log2) < n_slots) ++slot_log2;
    b.pshift = slot_log2 < kPartLog2 ? slot_log2 : kPartLog2;
    b.parts = (uint32_t)(n_slots >> b.pshift);
    b.pbits = slot_log2 - b.pshift;
    b.nblocks = std::max<int64_t>((n + kTile - 1) / kTile, 1);
    b.ovf_cap = n / 16 + 4096;
    b.scan_n = (int64_t)kBins * b.nblocks;
    const int64_t per = (b.scan_n + 1023) / 1024;
    b.scan_chunk = (per + kScanChunkAlign - 1) / kScanChunkAlign * kScanChunkAlign;
    b.scan_chunks = (int)((b.scan_n + b.scan_chunk - 1) / b.scan_chunk);
    return b;
}

}  // namespace

// Exclusive scan of data[0, n) in place; tmp: 1024 words of device scratch.
void launch_scan_u32_long(uint32_t* data, int64_t n, uint32_t* tmp, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t per = (n + 1023) / 1024;
    const int64_t chunk = (per + kScanChunkAlign - 1) / kScanChunkAlign * kScanChunkAlign;
    const int chunks = (int)((n + chunk - 1) / chunk);
    k_chunk_sums<<<chunks, kThreads, 0, s>>>(data, n, chunk, tmp);
    k_scan_small<<<1, 1024, 0, s>>>(tmp, chunks);
    k_chunk_scan<<<chunks, kThreads, 0, s>>>(data, n, chunk, tmp);
    note_launch(3);
}

size_t index_build_scratch_bytes(int64_t n, uint64_t n_slots) {
    const BuildPlan b = plan_for(n, n_slots);
    size_t t = 0;
    t += align_up((size_t)n * 8) * 2;  // hashes, ping-pong
    t += align_up((size_t)n * 4) * 2;  // rows, ping-pong
    t += align_up((size_t)b.scan_n * 4);
    t += align_up(1024 * 4);
    t += align_up(((size_t)b.parts + 1) * 4);
    t += align_up((size_t)b.ovf_cap * 8) * 2;
    t += 256;
    return t;
}

void launch_index_build(int Wd, const uint64_t* rows, int64_t n, HashView hv, uint64_t n_slots, void* scratch,
                        DevCounters* ctr, cudaStream_t s) {
    const BuildPlan b = plan_for(n, n_slots);
    char* p = (char*)scratch;
    uint64_t* h0 = (uint64_t*)p; p += align_up((size_t)n * 8);
    uint64_t* h1 = (uint64_t*)p; p += align_up((size_t)n * 8);
    uint32_t* r0 = (uint32_t*)p; p += align_up((size_t)n * 4);
    uint32_t* r1 = (uint32_t*)p; p += align_up((size_t)n * 4);
    uint32_t* hist = (uint32_t*)p; p += align_up((size_t)b.scan_n * 4);
    uint32_t* csum = (uint32_t*)p; p += align_up(1024 * 4);
    uint32_t* start = (uint32_t*)p; p += align_up(((size_t)b.parts + 1) * 4);
    uint64_t* ovf_e = (uint64_t*)p; p += align_up((size_t)b.ovf_cap * 8);
    uint64_t* ovf_h = (uint64_t*)p; p += align_up((size_t)b.ovf_cap * 8);
    unsigned long long* n_ovf = (unsigned long long*)p;
    cudaMemsetAsync(n_ovf, 0, sizeof(unsigned long long), s);

    // shared-memory limits above the 48 KB default (set per call: they are per device)
    const size_t scatter_smem = (size_t)kTile * 12;
    cudaFuncSetAttribute(k_part_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scatter_smem);
    cudaFuncSetAttribute(k_part_build, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 << kPartLog2);
    cudaFuncSetAttribute(k_part_scatter, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(k_part_build, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (n > 0) {
        const int g = grid_stride_blocks(n);
        switch (Wd) {
            case 1: k_build_hash<1><<<g, kThreads, 0, s>>>(rows, n, h0); break;
            case 2: k_build_hash<2><<<g, kThreads, 0, s>>>(rows, n, h0); break;
            default: k_build_hash<4><<<g, kThreads, 0, s>>>(rows, n, h0); break;
        }
        note_launch();
    }
    // order the records by partition: stable LSD passes over the partition index
    const uint64_t* hin = h0;
    const uint32_t* rin = nullptr;  // before the first pass, row = record index
    uint64_t* hout = h1;
    uint32_t* rout = r0;
    for (int dshift = 0; dshift < b.pbits && n > 0; dshift += kDigitBits) {
        k_part_hist<<<(unsigned)b.nblocks, kThreads, 0, s>>>(hin, n, hv.bucket_mask, b.pshift, dshift, hist,
                                                             b.nblocks);
        k_chunk_sums<<<b.scan_chunks, kThreads, 0, s>>>(hist, b.scan_n, b.scan_chunk, csum);
        k_scan_small<<<1, 1024, 0, s>>>(csum, b.scan_chunks);
        k_chunk_scan<<<b.scan_chunks, kThreads, 0, s>>>(hist, b.scan_n, b.scan_chunk, csum);
        k_part_scatter<<<(unsigned)b.nblocks, kSThreads, scatter_smem, s>>>(hin, rin, n, hv.bucket_mask, b.pshift,
                                                                           dshift, hist, b.nblocks, hout, rout);
        note_launch(5);
        uint64_t* hnext = (hin == h0) ? h0 : h1;  // the buffer just read becomes the next output
        uint32_t* rnext = (rout == r0) ? r1 : r0;
        hin = hout;
        rin = rout;
        hout = hnext;
        rout = rnext;
    }
    if (!rin) {  // one partition (or no rows): records in row order
        launch_iota(r0, n, s);
        rin = r0;
    }
    k_part_starts<<<grid_stride_blocks(n + 1), kThreads, 0, s>>>(hin, n, hv.bucket_mask, b.pshift, b.parts, start);
    k_part_build<<<b.parts, kThreads, (size_t)8 << b.pshift, s>>>(hin, rin, start, hv.bucket_mask, b.pshift,
                                                                  hv.max_probe * kBucketSlots, hv.slots, ovf_e, ovf_h,
                                                                  n_ovf, b.ovf_cap, ctr);
    k_part_overflow<<<64, kThreads, 0, s>>>(ovf_e, ovf_h, n_ovf, b.ovf_cap, hv.slots, n_slots,
                                            hv.max_probe * kBucketSlots, ctr);
    note_launch(3);
}

}  // namespace iqcc
