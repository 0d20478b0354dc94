// Internal declarations of libiqcc: device key helpers, the context, and the
// host-side launchers of every kernel.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/iqcc.h"

namespace iqcc {

// ----------------------------------------------------------------------------
// Keys on the device: a row is x[Wd] then z[Wd] (Wd = 1, 2 or 4 words, padded
// with zeros above the input's W), 16*Wd bytes, 16-byte aligned.
// ----------------------------------------------------------------------------

constexpr uint64_t kEmptySlot = ~0ull;        // hash slot never used
constexpr uint32_t kRowRemoved = 0xFFFFFFFFu; // compaction map entry of a removed row
constexpr int kBucketSlots = 4;               // 4 x 8-byte slots = one 32-byte sector

template <int W>
struct Key {
    uint64_t x[W];
    uint64_t z[W];
};

template <int W>
__device__ __forceinline__ Key<W> load_key(const uint64_t* __restrict__ rows, int64_t i) {
    Key<W> k;
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(rows + (size_t)i * 2 * W);
#pragma unroll
    for (int j = 0; j < W; ++j) {
        ulonglong2 v = __ldg(p + j);
        uint64_t a = v.x, b = v.y;
        // words 2j and 2j+1 of the row
        int w0 = 2 * j, w1 = 2 * j + 1;
        if (w0 < W) k.x[w0] = a; else k.z[w0 - W] = a;
        if (w1 < W) k.x[w1] = b; else k.z[w1 - W] = b;
    }
    return k;
}

template <>
__device__ __forceinline__ Key<1> load_key<1>(const uint64_t* __restrict__ rows, int64_t i) {
    ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(rows) + i);
    Key<1> k;
    k.x[0] = v.x;
    k.z[0] = v.y;
    return k;
}

template <int W>
__device__ __forceinline__ void store_key(uint64_t* rows, int64_t i, const Key<W>& k) {
    ulonglong2* p = reinterpret_cast<ulonglong2*>(rows + (size_t)i * 2 * W);
    uint64_t w[2 * W];
#pragma unroll
    for (int j = 0; j < W; ++j) { w[j] = k.x[j]; w[W + j] = k.z[j]; }
#pragma unroll
    for (int j = 0; j < W; ++j) p[j] = make_ulonglong2(w[2 * j], w[2 * j + 1]);
}

template <int W>
__device__ __forceinline__ bool key_equal(const Key<W>& a, const Key<W>& b) {
    uint64_t d = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) d |= (a.x[j] ^ b.x[j]) | (a.z[j] ^ b.z[j]);
    return d == 0;
}

template <int W>
__device__ __forceinline__ Key<W> key_xor(const Key<W>& a, const Key<W>& b) {
    Key<W> r;
#pragma unroll
    for (int j = 0; j < W; ++j) { r.x[j] = a.x[j] ^ b.x[j]; r.z[j] = a.z[j] ^ b.z[j]; }
    return r;
}

template <int W>
__device__ __forceinline__ int popc_and(const uint64_t* a, const uint64_t* b) {
    int s = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) s += __popcll(a[j] & b[j]);
    return s;
}

// Symplectic form: 1 when P(a) and P(b) anticommute.
template <int W>
__device__ __forceinline__ int anticommutes(const Key<W>& a, const Key<W>& b) {
    uint64_t v = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) v ^= (a.x[j] & b.z[j]) ^ (a.z[j] & b.x[j]);
    return __popcll(v) & 1;
}

// For anticommuting Hermitian strings T and P with Q = T xor P:
//   i T P = s Q, s = +1 when e = 3 and -1 when e = 1, where
//   e = popc(xT&zT) + popc(xP&zP) + 2 popc(zT&xP) - popc(xQ&zQ)  (mod 4).
// (From P(x,z) = i^{popc(x&z)} X^x Z^z and Z^a X^b = (-1)^{popc(a&b)} X^b Z^a.)
template <int W>
__device__ __forceinline__ int product_sign(const Key<W>& t, int yP, const Key<W>& p, const Key<W>& q) {
    int e = popc_and<W>(t.x, t.z) + yP + 2 * popc_and<W>(t.z, p.x) - popc_and<W>(q.x, q.z);
    return ((e & 3) == 3) ? 1 : -1;
}

// Key hash: a multiply-xorshift chain over the 2W words, finished with the
// 64-bit fmix of MurmurHash3.  Low bits pick the bucket; the top 24 bits are
// the fingerprint kept in index entries (the DIS group table keeps the top 32).
template <int W>
__device__ __forceinline__ uint64_t hash_key(const Key<W>& k) {
    uint64_t h = 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        h = (h ^ k.x[j]) * 0xBF58476D1CE4E5B9ull;
        h ^= h >> 31;
        h = (h ^ k.z[j]) * 0x94D049BB133111EBull;
        h ^= h >> 29;
    }
    h ^= h >> 33;
    h *= 0xFF51AFD7ED558CCDull;
    h ^= h >> 33;
    h *= 0xC4CEB9FE1A85EC53ull;
    h ^= h >> 33;
    return h;
}

// Hash of the pair key of T for generator P whose lowest set bit is bit
// `mask` of word `word` (0..2W-1, x words first): of T and its partner
// T xor P, the one with that bit clear (exactly one of them), so the same for
// both members of a pair.  Its top bits pick the dress bin.
template <int W>
__device__ __forceinline__ uint64_t pair_hash(const Key<W>& t, const Key<W>& p, int word, uint64_t mask) {
    uint64_t v = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        if (word == j) v = t.x[j];
        if (word == W + j) v = t.z[j];
    }
    const uint64_t flip = (v & mask) ? ~0ull : 0ull;
    Key<W> k;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        k.x[j] = t.x[j] ^ (p.x[j] & flip);
        k.z[j] = t.z[j] ^ (p.z[j] & flip);
    }
    return hash_key<W>(k);
}

// Device-side counters shared by the kernels of one call.
struct DevCounters {
    unsigned long long n_new;      // rows appended by a dress
    unsigned long long n_anti;     // anticommuting rows seen by a dress
    unsigned long long n_groups;   // DIS groups / compaction output
    unsigned long long aux;        // scratch counter
    int err;                       // iqcc_status set by a kernel (first error wins)
    int err_where;                 // which kernel
    int wait_limit;                // polls a device wait makes before it reports IQCC_ERR_TIMEOUT
    int pad;
};
// Bytes of DevCounters cleared between calls (everything before wait_limit).
constexpr size_t kCountersClear = offsetof(DevCounters, wait_limit);
constexpr int kDefaultWaitLimit = 1 << 24;  // polls of about 32-64 ns: a wait gives up after about a second

// First error wins; `where` names the raising site.
__device__ __forceinline__ void set_error(DevCounters* ctr, int code, int where) {
    if (atomicCAS(&ctr->err, 0, code) == 0) ctr->err_where = where;
}

// Index entries (one 8-byte slot each): bits 63..40 are the top 24 bits of the
// key's hash (a fingerprint checked before the key itself is read), bits 39..32
// the entry's distance in buckets from its home bucket (so an entry's home is
// known without its key), bits 31..0 the row.  Rows stay below 0xFFFFFFFE, so
// no entry equals kEmptySlot.
constexpr uint64_t kFpMask = 0xFFFFFF0000000000ull;
constexpr int kMaxProbeLimit = 256;  // displacements fit 8 bits

__host__ __device__ __forceinline__ uint64_t make_entry(uint64_t hv, uint32_t row, uint64_t disp) {
    return (hv & kFpMask) | (disp << 32) | (uint64_t)row;
}
__host__ __device__ __forceinline__ bool fp_match(uint64_t entry, uint64_t hv) {
    return ((entry ^ hv) & kFpMask) == 0;
}
__host__ __device__ __forceinline__ uint32_t entry_disp(uint64_t entry) { return (uint32_t)(entry >> 32) & 0xFFu; }

// Hash table view.
struct HashView {
    uint64_t* slots;
    uint64_t bucket_mask;  // number of buckets - 1 (buckets are 4 slots)
    int max_probe;
};

// Generator of one dress / A,B,C pass.
template <int W>
struct Gen {
    Key<W> p;
    int yP;          // popc(xP & zP) mod 4
    int top_word;    // word index (0..2W-1, x words first) of P's lowest set bit
    uint64_t top_mask;  // that bit
    double cos_t, sin_t;
};

// Generator of a device-layout key pkey (x words then z words): P, its Y
// count mod 4, the word and bit of P's lowest set bit (first non-zero word,
// x words first), and the rotation.
template <int W>
inline Gen<W> make_gen(const uint64_t* pkey, double cos_t, double sin_t) {
    Gen<W> g{};
    int y = 0;
    g.top_word = -1;
    for (int j = 0; j < W; ++j) {
        g.p.x[j] = pkey[j];
        g.p.z[j] = pkey[W + j];
        y += __builtin_popcountll(pkey[j] & pkey[W + j]);
    }
    for (int w = 0; w < 2 * W && g.top_word < 0; ++w)
        if (pkey[w]) {
            g.top_word = w;
            g.top_mask = pkey[w] & (~pkey[w] + 1);
        }
    if (g.top_word < 0) {
        g.top_word = 0;
        g.top_mask = 0;
    }
    g.yP = y & 3;
    g.cos_t = cos_t;
    g.sin_t = sin_t;
    return g;
}

// Batches of independent Hamiltonians (one word per x and z): problem b's
// strings carry b in z bits kBatchTagShift.. (Z letters on virtual qubits).
constexpr int kBatchTagShift = 48;
constexpr int kMaxBatch = 2048;

// ----------------------------------------------------------------------------
// Context
// ----------------------------------------------------------------------------

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace iqcc

struct iqcc_ctx {
    int n = 0;            // qubits
    int W = 0;            // host words per x / z vector
    int Wd = 0;           // device words (1, 2, 4)
    int64_t capacity = 0; // admission limit (rows)
    int max_probe = 64;
    int device = 0;       // the CUDA device the context lives on
    cudaStream_t stream = nullptr;
    void* (*alloc)(size_t, void*) = nullptr;
    void (*dfree)(void*, void*) = nullptr;
    void* alloc_user = nullptr;

    int64_t M = 0;                 // live rows
    int64_t rows_alloc = 0;        // rows allocated in the key/coef buffers
    iqcc::Buf keys, coef;
    iqcc::Buf keys2, coef2;        // the other row buffer: a dress writes H there and the two swap
    iqcc::Buf hash;                // slots of the key index (partitioned dressing and batches only)
    uint64_t hash_slots = 0;       // active slots (power of two)
    bool index_valid = false;      // the index holds exactly rows [0, M)
    iqcc::Buf dropflags;           // a deferred term-limit cut: 1 for the rows it keeps
    bool pending = false;          // dropflags applies to rows [0, M); the next dress drops the rest
    int64_t live = 0;              // rows kept by the pending cut (M when none is pending)
    iqcc::Buf pairbuf;             // dress bins: [0] = 0, then per bin its count, start, end
    bool pair_ready = false;       // pairbuf holds the bin counts of pair_key's dress of the current H
    int pair_log2 = 0;
    int64_t pair_n_anti = 0;       // rows counted into those bins
    uint64_t pair_key[8] = {0};    // device-layout key of that generator
    iqcc::Buf counters;            // DevCounters
    iqcc::DevCounters* h_counters = nullptr;  // pinned host mirror
    iqcc::Buf scratch;             // general scratch (grows)
    iqcc::Buf aux;                 // second scratch for sizes known only mid-call
    long long launch_base = 0;     // library launch count at the last stats reset
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    bool broken = false;
    std::string err;
    iqcc_stats stats{};
    iqcc::Buf model;               // learned screening weights (device layout), when set
    iqcc::Buf screen_rank;         // learned screening: per-row keys and the <sigma> table
    double screen_floor = 0.5;     // learned term limit: share kept by largest |C| first
    int select_guess = -1;         // first-level digit of the last term-limit select (-1: none yet)
    double bin_slack = 0.25;       // fixed dress bins: relative slack over the mean count
    int bin_slack_rows = 32;       //   and rows added to it

    uint64_t* rows() const { return (uint64_t*)keys.p; }
    double* c() const { return (double*)coef.p; }
};

namespace iqcc {

// ----------------------------------------------------------------------------
// Host launchers (defined in the k_*.cu files).  All run on ctx->stream.
// ----------------------------------------------------------------------------

int device_words(int n);
int current_device();
int sm_count();  // of the current device
// True on the first call for the current device with this `seen` mask, and
// for every call on devices past the 64th: per-device set-up such as
// cudaFuncSetAttribute, whose settings belong to each device's context.
bool first_on_device(std::atomic<unsigned long long>* seen);
void note_launch();     // counts kernel launches of the library (all launchers call it)
void note_launch(int k);  // k launches
long long launches();

// k_build.cu: index build without global atomics on the table (partitioned in
// shared memory); writes every slot, so no clear is needed first.
size_t index_build_scratch_bytes(int64_t n, uint64_t n_slots);
// exclusive scan of a long u32 array in place (tmp: 1024 words of device scratch)
void launch_scan_u32_long(uint32_t* data, int64_t n, uint32_t* tmp, cudaStream_t s);
void launch_index_build(int Wd, const uint64_t* rows, int64_t n, HashView h, uint64_t n_slots, void* scratch,
                        DevCounters* ctr, cudaStream_t s);
// k_grad.cu: adjoint of the dressed QMF energy.  tab: energy_grad_table_doubles(n)
// per-qubit values; partials: [blocks][energy_grad_cols(n)]; the column sums go
// through launch_grad_combine to out[2n + 3] = (dE/dtheta, dE/dphi, A, B, C).
int energy_grad_blocks();
int energy_grad_table_doubles(int n);
int energy_grad_cols(int n);
void launch_grad_tables(const double* theta, const double* phi, int n, double* tab, cudaStream_t s);
void launch_energy_grad(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* pkey,
                        bool has_gen, double cos_t, double sin_t, const double* tab, int n, const uint64_t* occ_words,
                        bool basis, double* partials, int blocks, cudaStream_t s);
void launch_grad_combine(const double* sums, const double* tab, int n, double* out, cudaStream_t s);

// k_sortdress.cu: expansion of rows through a group of up to max_fuse()
// generators (pkeys: k device-layout keys of 2*Wd words, host memory; tau: host).
int max_fuse();
void launch_expand_count(int Wd, const uint64_t* rows, int64_t M, const uint64_t* pkeys, const double* tau, int k,
                         unsigned long long* total, cudaStream_t s);
void launch_expand_emit(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* pkeys,
                        const double* tau, int k, uint64_t* out_rows, double* out_coef, unsigned long long* next,
                        int64_t cap, DevCounters* ctr, cudaStream_t s);

// k_batch.cu: per-problem reductions of a batch (z-eigenstate references).
// partials: [blocks][B] (energy), [blocks][3B] (A, B, C); counts[B] accumulate.
void launch_seg_energy(const uint64_t* rows, const double* coef, int64_t M, const uint64_t* occ, int B,
                       double* partials, unsigned long long* counts, int blocks, cudaStream_t s);
void launch_seg_dis_group(const uint64_t* rows, const double* coef, int64_t M, const uint64_t* occ, int B,
                          uint64_t* slots, double* gsum, uint64_t bucket_mask, int max_probe, DevCounters* ctr,
                          int blocks, cudaStream_t s);
void launch_seg_best(const uint64_t* slots, const double* gsum, uint64_t n_slots, int B,
                     unsigned long long* best_coarse, unsigned long long* best_key, double* best_g, int blocks,
                     cudaStream_t s);
void launch_seg_abc(const uint64_t* rows, const double* coef, int64_t M, const uint64_t* occ, int B,
                    const unsigned long long* best_key, double* partials, int blocks, cudaStream_t s);
void launch_seg_tau(const double* abc, const unsigned long long* best_key, int B, double* tau, Gen<1>* gens,
                    cudaStream_t s);
// partitioned dressing (k_dress.cu): the anticommuting rows of P appended to
// ox/oz [.][Wout] and oc (at most cap; the count in *n_out), and the dress of
// the local rows given the peer's anticommuting rows (prow/pcoef, indexed by hp)
void launch_cross_rows(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* pkey, int Wout,
                       int64_t cap, uint64_t* ox, uint64_t* oz, double* oc, unsigned long long* n_out,
                       cudaStream_t s);
void launch_cross_dress(int Wd, const uint64_t* rows, double* coef, int64_t M, const uint64_t* pkey, double cos_t,
                        double sin_t, HashView h, HashView hp, const uint64_t* prow, const double* pcoef,
                        int64_t n_peer, DevCounters* ctr, cudaStream_t s);

// k_screen.cu: learned term screening (features, perceptron scores).  gsup:
// union of the generators' supports (Wd words); ev: per-qubit <sigma> at
// stride ts (the energy-gradient table).  model: screen_model_bytes() on the device.
int screen_features();
// out[i] = in[perm[i]] for rows of `width` bytes (a multiple of 4)
void launch_gather_bytes(const void* in, const uint32_t* perm, int64_t n, int width, void* out, cudaStream_t s);
size_t screen_model_bytes();
void pack_screen_model(const float* w1, const float* b1, const float* w2, const float* b2, const float* w3, float b3,
                       unsigned char* out);
void launch_term_features(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* gsup,
                          const double* ev, int ts, int n, float* out, cudaStream_t s);
void launch_mlp_score(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* gsup,
                      const double* ev, int ts, int n, const void* model, float* score, double* rank,
                      cudaStream_t s);
// k_sortdress.cu: energy of every row after k <= max_fuse() generators (tab: <sigma> at stride ts)
void launch_future_energy(int Wd, const uint64_t* rows, int64_t M, const uint64_t* pkeys, const double* tau, int k,
                          const double* tab, int ts, int n, double* out, cudaStream_t s);

// k_pairjoin.cu: dress by pair partition (histogram, split, shared-memory join).
// The split works on tiles of kDressTile rows (256 threads, 4 rows each); the
// counting pass before it (launch_pair_hist, or the A, B, C pass of
// iqcc_iterate) counts per tile the rows the split keeps, so that each tile's
// output offset is known in advance.
constexpr int kDressTile = 1024;
struct PairDress {
    int Wd;
    const uint64_t* pkey;    // host, device-layout key of the one generator (gens == nullptr)
    const Gen<1>* gens;      // device, per-problem generators of a batch (Wd == 1), or nullptr
    int B;
    double cos_t, sin_t;
};
int pair_bins_log2(int64_t M);
uint32_t pair_bins_per_block(int64_t n_anti, int log2_bins);
// counts: [2^log2_bins] zeroed; adds each anticommuting row to its bin and the total to ctr->n_anti;
// tile_kept[t]: the rows of tile t the split keeps (commuting, live).
// live (may be NULL): rows with live[i] == 0 are dropped (a pending term-limit cut), here and in the split.
void launch_pair_hist(const PairDress& d, const uint64_t* rows, int64_t M, int log2_bins, uint32_t* counts,
                      uint32_t* tile_kept, DevCounters* ctr, cudaStream_t s, const uint8_t* live = nullptr);
// From rows/coef (M rows) into rows_out/coef_out: the kept rows of tile t from tile_off[t] on (compact);
// rk [.][2 Wd] keys and rc [.] coefficients of the anticommuting rows, by bin (scatter).  cap == 0:
// cursor holds the bin starts (scanned exact counts) in, bin ends out.  cap > 0: bins of cap rows
// (bin b at b cap), cursor zeroed in, rows received per bin out; rows past a full bin are counted in
// ctr->aux and dropped (the caller then redoes the dress with exact counts).
void launch_pair_split(const PairDress& d, bool compact, bool scatter, const uint64_t* rows, const double* coef,
                       int64_t M, int log2_bins, uint32_t* cursor, uint32_t cap, uint64_t* rk, double* rc,
                       const uint32_t* tile_off, uint64_t* rows_out, double* coef_out, DevCounters* ctr,
                       cudaStream_t s, const uint8_t* live = nullptr);
// start: [2^log2_bins + 1] bin starts (cap == 0) or the rows each fixed-size bin received (cap > 0,
// one bin per block); rows without a partner counted in ctr->n_new; with `write` the dressed rows and
// appended partners are written to rows/coef from row *kept + (*out_cursor, zeroed) on
void launch_pair_join(const PairDress& d, bool write, const uint64_t* rk, const double* rc, const uint32_t* start,
                      int log2_bins, uint32_t bins_per_block, uint64_t* rows, double* coef, const uint32_t* kept,
                      unsigned long long* out_cursor, DevCounters* ctr, cudaStream_t s, uint32_t cap = 0);

// Bins filled from two partitions of one Hamiltonian (one generator, d.gens == nullptr): the join
// writes each output row to the partition owning its key.  mask, aval: device-layout keys; a key k
// belongs to partition 0 iff (k & mask) == aval.
struct PairTwo {
    uint64_t mask[8], aval[8];
    uint64_t* rows[2];
    double* coef[2];
    const uint32_t* kept[2];
    unsigned long long* cursor[2];
};
void launch_pair_join2(const PairDress& d, const uint64_t* rk, const double* rc, const uint32_t* start,
                       int log2_bins, uint32_t bins_per_block, const PairTwo& t, DevCounters* ctr, cudaStream_t s);

// tile_kept[t]: flagged rows in tile t of kDressTile rows (an out-of-place compaction's offsets,
// after a scan, for launch_pair_split with a zero generator and the flags as live rows).
void launch_flag_tiles(const uint8_t* flags, int64_t n, uint32_t* tile_kept, cudaStream_t s);
// Load of rows in any order (k_pairjoin.cu): the distinct keys of rows[0, n) with their coefficients
// summed in input order, non-zero sums written to rows_out / c_out from *out_cursor (zeroed) on, in
// bin order.  Three phases: 0 counts rows per bin into counts[1..2^L] (zeroed, counts[0] = 0);
// then the caller scans counts[1..2^L] (bin starts) and checks that no group of bins_per_block bins
// holds more than 4096 rows; 1 copies rows into their bins (rk [n][2 Wd], rc, ri = input index;
// counts[1..] advance to bin ends, so counts[b] is bin b's start); 2 joins each group of bins.
void launch_key_group(int Wd, const uint64_t* rows, const double* coef, int64_t n, int log2_bins, int phase,
                      uint32_t* counts, uint64_t* rk, double* rc, uint32_t* ri, uint32_t bins_per_block,
                      uint64_t* rows_out, double* c_out, unsigned long long* out_cursor, DevCounters* ctr,
                      cudaStream_t s);
constexpr int kKeyJoinCap = 4096;  // rows one key-join block holds

// k_dress.cu: the key index (partitioned dress only)
void launch_hash_clear(HashView h, uint64_t slots, cudaStream_t s);
void launch_hash_insert(int Wd, const uint64_t* rows, int64_t lo, int64_t hi, HashView h,
                        DevCounters* ctr, cudaStream_t s);

// k_expect.cu
int expect_blocks();
// Fills partials[block][3] with (A, B, C) sums; pkey may be all-zero (energy).
// With `pair` the same pass also counts P's anticommuting rows by dress bin
// (launch_pair_hist's output, for the dress by P that follows).
struct PairHistOut {
    uint32_t* counts;     // [2^log2_bins], zeroed
    uint32_t* tile_kept;  // [ceil(M / kDressTile)]: rows per tile the split keeps (commuting, live)
    int log2_bins;
    DevCounters* ctr;     // n_anti (zeroed) receives the total
};
// live (may be NULL: every row): rows with live[i] == 0 are skipped (a pending term-limit cut).
void launch_abc(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* pkey,
                bool basis, const uint64_t* occ, const double* tables, int n_groups, double* partials,
                cudaStream_t s, const PairHistOut* pair = nullptr, const uint8_t* live = nullptr);
void launch_reduce3(const double* partials, int n, double* out3, cudaStream_t s);
void launch_qmf_tables(const double* theta, const double* phi, int n, int n_groups, double* tables,
                       cudaStream_t s);
// k_disgroup.cu: DIS candidates by partition.  launch_flip_hist counts the rows
// with a non-empty flip set into 2^log2_bins bins (counts zeroed; total to
// ctr->aux); after an exclusive scan of counts, launch_flip_group copies them
// into their bins (flip sets and, when `values`, z-eigenstate
// contributions) and writes one (flip set, summed
// contribution) per distinct flip set to gkeys [.][Wd] / gsum, counted in
// ctr->n_groups (at most max_groups).  arr: [0] = 0, then the bin starts;
// rr: flip_record_bytes(Wd) per row with a non-empty flip set.
void launch_flip_hist(int Wd, const uint64_t* rows, int64_t M, int log2_bins, uint32_t* counts, DevCounters* ctr,
                      cudaStream_t s);
size_t flip_record_bytes(int Wd);
void launch_flip_group(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* occ_words,
                       bool values, int log2_bins, uint32_t* arr, uint64_t* rr, int64_t n_flip, uint64_t* gkeys,
                       double* gsum, int64_t max_groups, DevCounters* ctr, cudaStream_t s);
// General-angle gradients of K candidates: partials[block][K].
void launch_grad_general(int Wd, const uint64_t* rows, const double* coef, int64_t M,
                         const uint64_t* cand, int K, const double* tables, int n_groups,
                         double* partials, int n_blocks, cudaStream_t s);
void launch_reduce_cols(const double* partials, int rows, int cols, double* out, cudaStream_t s);

// k_sort.cu
struct SortPlan {
    int n_words;          // key words per element (stride in the key array)
    int order[9];         // word indices from most to least significant
    int n_order;
};
// Indirect stable LSD radix sort of perm[0..n) by keys[perm[i]*stride + order[..]].
// perm_alt is scratch of the same size; the result ends in *result (one of the two).
void radix_sort_indirect(const uint64_t* keys, int stride, const SortPlan& plan, uint32_t* perm,
                         uint32_t* perm_alt, int64_t n, uint32_t** result, void* scratch,
                         size_t scratch_bytes, cudaStream_t s);
size_t radix_sort_scratch_bytes(int64_t n);
void launch_iota(uint32_t* p, int64_t n, cudaStream_t s);

// compaction: out[rank] = in[i] for flags[i] != 0 (stable); count to *ctr_count (device).
size_t compact_scratch_bytes(int64_t n);
// k_keysort.cu: rows [0, n) and coefficients sorted in canonical order, the
// first k written as x [k][W], z [k][W], coef [k] into dst_* when all three
// are device-writable addresses, else inside scratch (pointers out).
size_t export_sort_scratch_bytes(int Wd, int64_t n);
void launch_export_sort(int W, int Wd, const uint64_t* rows, const double* coef, int64_t n, int64_t k, void* scratch,
                        uint64_t* dst_x, uint64_t* dst_z, double* dst_c, uint64_t** out_x, uint64_t** out_z,
                        double** out_c, cudaStream_t s);
// adds to *count the consecutive pairs not strictly increasing in canonical order
void launch_order_violations(int Wd, const uint64_t* rows, int64_t n, unsigned long long* count, cudaStream_t s);
void launch_compact_rows(int Wd, const uint8_t* flags, const uint64_t* rows_in, const double* c_in,
                         uint64_t* rows_out, double* c_out, int64_t n, void* scratch,
                         unsigned long long* count, cudaStream_t s);

// single-pass in-place stable compaction of rows/coef by flags; kept count to *count
size_t compact_inplace_scratch_bytes(int64_t n);
// new_row (may be NULL): per old row, its new index or kRowRemoved
void launch_compact_inplace(int Wd, const uint8_t* flags, uint64_t* rows, double* coef, int64_t n, void* scratch,
                            unsigned long long* count, DevCounters* ctr, cudaStream_t s,
                            uint32_t* new_row = nullptr);

// one bounded wait on *word (zero, never written): records IQCC_ERR_TIMEOUT once ctr->wait_limit is spent
void launch_wait_selftest(const unsigned long long* word, DevCounters* ctr, cudaStream_t s);

// DIS top-k: coarse |g| radix select, collect, sort of the collected subset
void launch_coarse_digit_hist(const double* g, int64_t G, int shift, uint64_t prefix, uint64_t prefix_mask,
                              unsigned long long* hist, cudaStream_t s);
void launch_collect_ge(const double* g, int64_t G, uint64_t t, uint32_t* idx, int64_t cap, unsigned long long* count,
                       cudaStream_t s);
void launch_dis_sort_keys_sub(int Wd, const uint64_t* gkeys, const double* gsum, const uint32_t* idx, int64_t k,
                              uint64_t* skeys, cudaStream_t s);

// load: pack host-layout x/z into rows, sum runs after the sort
// host layout to device rows; keys with bits in hi_mask of their last word counted in *bad (may be NULL)
void launch_pack_rows(int W, int Wd, const uint64_t* x, const uint64_t* z, uint64_t* rows, int64_t n,
                      cudaStream_t s, uint64_t hi_mask = 0, unsigned long long* bad = nullptr);
void launch_unpack_rows(int W, int Wd, const uint64_t* rows, const double* coef, const uint32_t* perm,
                        uint64_t* x, uint64_t* z, double* c, int64_t n, cudaStream_t s);
void launch_sum_runs(int Wd, const uint64_t* rows, const double* coef, const uint32_t* perm, int64_t n,
                     uint8_t* flags, uint64_t* rows_out_gather, double* c_out_gather, cudaStream_t s,
                     bool keep_zeros = false);
void launch_gather_rows(int Wd, const uint64_t* rows, const double* coef, const uint32_t* perm,
                        int64_t n, uint64_t* rows_out, double* c_out, cudaStream_t s);

// prune
void launch_prune_flags(const double* coef, int64_t n, double eps, uint8_t* flags,
                        unsigned long long* count, cudaStream_t s);
// histogram of one 8-bit digit of |c| bits among kept rows whose higher digits equal prefix
void launch_abs_digit_hist(const double* coef, const uint8_t* flags, int64_t n, int shift,
                           uint64_t prefix, uint64_t prefix_mask, unsigned long long* hist,
                           cudaStream_t s);
// flags: 1 if |c| bits > t; ties (== t) are listed into tie_idx (count in *tie_count)
void launch_budget_flags(const double* coef, uint8_t* flags, int64_t n, uint64_t t_bits,
                         uint32_t* tie_idx, unsigned long long* tie_count, cudaStream_t s);
void launch_set_flags(const uint32_t* idx, int64_t k, uint8_t* flags, cudaStream_t s);
// term-limit select with 12-bit digits, then an exact sort of the threshold bucket
void launch_abs_digit_hist12(const double* coef, const uint8_t* flags, int64_t n, int shift, uint64_t prefix,
                             uint64_t prefix_mask, unsigned long long* hist, cudaStream_t s);
// The first two select levels in one pass: hist1 (4096, zeroed) of the digit at shift1 of every kept
// row, hist2 (4096, zeroed) of the digit at shift2 of the kept rows whose first digit is `guess`.
void launch_abs_digit_hist12x2(const double* coef, const uint8_t* flags, int64_t n, int shift1, int shift2,
                               unsigned guess, unsigned long long* hist1, unsigned long long* hist2, cudaStream_t s);
void launch_bucket_flags(const double* coef, uint8_t* flags, int64_t n, uint64_t prefix, uint64_t prefix_mask,
                         uint32_t* cand, unsigned long long* n_cand, cudaStream_t s);
// |c| bit patterns (as doubles) of the kept rows in a select bucket, appended to
// vals (at most cap; *n_vals counts all)
void launch_bucket_values(const double* coef, const uint8_t* flags, int64_t n, uint64_t prefix, uint64_t prefix_mask,
                          double* vals, unsigned long long* n_vals, int64_t cap, cudaStream_t s);
// rank[i] = boost where flags[i] and the |c| bits reach t_bits
void launch_boost_rank(const double* coef, const uint8_t* flags, int64_t n, uint64_t t_bits, double boost, double* rank,
                       cudaStream_t s);
// flags[i] = |c| bits above the bucket (every row live); bucket rows listed in cand
void launch_cut_flags(const double* coef, uint8_t* flags, int64_t n, uint64_t prefix, uint64_t prefix_mask,
                      uint32_t* cand, unsigned long long* n_cand, cudaStream_t s);
void launch_candidate_keys(int Wd, const uint64_t* rows, const double* coef, const uint32_t* cand, int64_t k,
                           uint64_t* skeys, cudaStream_t s);
void launch_set_flags_sorted(const uint32_t* cand, const uint32_t* order, int64_t k, uint8_t* flags, cudaStream_t s);
// out[i] = keys[order[i] * stride]: the first word of each key in sorted order
void launch_gather_word(const uint64_t* keys, int stride, const uint32_t* order, int64_t n, uint64_t* out,
                        cudaStream_t s);
// cand: candidates of all parts concatenated (part p's at [offs[p], offs[p + 1])); flags: device array of
// the parts' flag arrays; the first k in `order` set in their owner's flags.
void launch_set_flags_sorted_parts(const uint32_t* cand, const uint32_t* order, int64_t k, const int64_t* offs,
                                   uint8_t* const* flags, int n_parts, cudaStream_t s);

// DIS candidate keys for the sort: [coarse |g| complement, x words...]
void launch_dis_sort_keys(int Wd, const uint64_t* gkeys, const double* gsum, int64_t G, uint64_t* skeys,
                          cudaStream_t s);
// candidate i is group perm[i] (or idx[perm[i]] when idx is given)
void launch_dis_export(int W, int Wd, const uint64_t* gkeys, const double* gsum, const uint32_t* perm,
                       const uint32_t* idx, int64_t k, uint64_t* ox, uint64_t* oz, double* og, cudaStream_t s);

}  // namespace iqcc
