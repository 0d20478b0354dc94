// C ABI of libiqcc: context management and the host-side sequencing of the
// kernels in k_dress.cu, k_expect.cu and k_sort.cu.  Declarations and the
// contract of every entry point are in include/iqcc.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "iqcc_internal.cuh"

using namespace iqcc;

namespace {

thread_local std::string g_last_error = "no error";

constexpr double kPi = 3.141592653589793;

iqcc_status fail(iqcc_ctx* ctx, iqcc_status st, const std::string& msg) {
    if (ctx) {
        ctx->err = msg;
        if (st == IQCC_ERR_CUDA || st == IQCC_ERR_HASH_FULL || st == IQCC_ERR_TIMEOUT) ctx->broken = true;
    } else {
        g_last_error = msg;
    }
    return st;
}

iqcc_status fail_cuda(iqcc_ctx* ctx, cudaError_t e, const char* what, int line) {
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s at abi.cu:%d", (int)e, cudaGetErrorString(e), what, line);
    return fail(ctx, IQCC_ERR_CUDA, buf);
}

#define CK(call)                                                        \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return fail_cuda(ctx, e_, #call, __LINE__); \
    } while (0)

#define CK_LAUNCH() CK(cudaGetLastError())

// As CK / CK_LAUNCH for a named context (calls over several contexts).
#define CK_CTX(c, call)                                                     \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return fail_cuda((c), e_, #call, __LINE__);  \
    } while (0)
#define CK_LAUNCH_CTX(c) CK_CTX((c), cudaGetLastError())

#define GUARD(ctx)                                                                 \
    do {                                                                           \
        if (!(ctx)) return fail(nullptr, IQCC_ERR_ARG, "null context");            \
        if ((ctx)->broken) return IQCC_ERR_STATE;                                  \
    } while (0)

void* dalloc(iqcc_ctx* ctx, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (ctx->alloc) {
        p = ctx->alloc(bytes, ctx->alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dfree(iqcc_ctx* ctx, void* p) {
    if (!p) return;
    if (ctx->dfree) ctx->dfree(p, ctx->alloc_user);
    else cudaFree(p);
}

void release(iqcc_ctx* ctx, Buf& b) {
    dfree(ctx, b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// Make b hold at least `bytes`; contents are not kept.
bool ensure(iqcc_ctx* ctx, Buf& b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return true;
    size_t want = std::max(bytes, b.bytes + b.bytes / 2);
    cudaStreamSynchronize(ctx->stream);
    void* p = dalloc(ctx, want);
    if (!p) {
        p = dalloc(ctx, bytes);
        want = bytes;
    }
    if (!p) return false;
    release(ctx, b);
    b.p = p;
    b.bytes = want;
    return true;
}

// Grow b to at least `bytes`, keeping the first `keep` bytes.
bool grow_keep(iqcc_ctx* ctx, Buf& b, size_t bytes, size_t keep) {
    if (b.bytes >= bytes && b.p) return true;
    void* p = dalloc(ctx, bytes);
    if (!p) return false;
    if (keep && b.p) {
        if (cudaMemcpyAsync(p, b.p, keep, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            dfree(ctx, p);
            return false;
        }
    }
    cudaStreamSynchronize(ctx->stream);
    release(ctx, b);
    b.p = p;
    b.bytes = bytes;
    return true;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Bump allocator over ctx->scratch: first compute the total with a dry run of
// take(), then ensure() and carve.
struct Carver {
    char* base = nullptr;
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        T* p = (T*)(base ? base + off : nullptr);
        off += align256(count * sizeof(T) + 1);
        return p;
    }
};

// The real carve must end inside the scratch allocation (guards the dry-run sizing).
bool carve_fits(const iqcc_ctx* ctx, const Carver& cv) { return cv.off <= ctx->scratch.bytes; }

size_t row_bytes(const iqcc_ctx* ctx) { return (size_t)16 * ctx->Wd; }

HashView hash_view(const iqcc_ctx* ctx) {
    HashView h;
    h.slots = (uint64_t*)ctx->hash.p;
    h.bucket_mask = ctx->hash_slots / kBucketSlots - 1;
    h.max_probe = ctx->max_probe;
    return h;
}

DevCounters* dctr(iqcc_ctx* ctx) { return (DevCounters*)ctx->counters.p; }

// Terms of H: the rows, less those a pending term-limit cut drops.
int64_t live_terms(const iqcc_ctx* ctx) { return ctx->pending ? ctx->live : ctx->M; }

// The pending cut's flags for kernels that skip dropped rows (NULL: none pending).
const uint8_t* live_flags(const iqcc_ctx* ctx) { return ctx->pending ? (const uint8_t*)ctx->dropflags.p : nullptr; }

iqcc_status read_counters(iqcc_ctx* ctx) {
    CK(cudaMemcpyAsync(ctx->h_counters, ctx->counters.p, sizeof(DevCounters), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const DevCounters& c = *ctx->h_counters;
    if (c.err) {
        char buf[160];
        snprintf(buf, sizeof buf, "device error %d raised by kernel site %d", c.err, c.err_where);
        return fail(ctx, (iqcc_status)c.err, buf);
    }
    return IQCC_OK;
}

uint64_t pow2_at_least(uint64_t v) {
    uint64_t p = 1024;
    while (p < v) p <<= 1;
    return p;
}

// (Re)build the index over rows [0, M) with `slots` slots.
iqcc_status rebuild_hash(iqcc_ctx* ctx, uint64_t slots) {
    if (slots != ctx->hash_slots || !ctx->hash.p) {
        release(ctx, ctx->hash);
        ctx->hash_slots = 0;
        if (!ensure(ctx, ctx->hash, slots * sizeof(uint64_t))) return fail(ctx, IQCC_ERR_OOM, "hash allocation failed");
        ctx->hash_slots = slots;
    }
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    HashView h = hash_view(ctx);
#ifndef IQCC_INDEX_BUILD_CAS
    // partitioned build (k_build.cu) in the auxiliary buffer; CAS inserts into a
    // cleared table where that buffer cannot grow
    if (ensure(ctx, ctx->aux, index_build_scratch_bytes(ctx->M, ctx->hash_slots))) {
        launch_index_build(ctx->Wd, ctx->rows(), ctx->M, h, ctx->hash_slots, ctx->aux.p, dctr(ctx), ctx->stream);
        CK_LAUNCH();
    } else
#endif
    {
        launch_hash_clear(h, ctx->hash_slots, ctx->stream);
        CK_LAUNCH();
        launch_hash_insert(ctx->Wd, ctx->rows(), 0, ctx->M, h, dctr(ctx), ctx->stream);
        CK_LAUNCH();
    }
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    ctx->stats.hash_ms += ms;
    ctx->stats.hash_rebuilds++;
    ctx->stats.hash_slots = (int64_t)ctx->hash_slots;
    return read_counters(ctx);
}

// Rows able to hold `rows_needed` rows (current rows kept).
iqcc_status reserve_rows(iqcc_ctx* ctx, int64_t rows_needed) {
    if (rows_needed > ctx->rows_alloc) {
        int64_t want = std::max<int64_t>(rows_needed, ctx->rows_alloc + ctx->rows_alloc / 2);
        want = std::min<int64_t>(want, ctx->capacity);
        want = std::max<int64_t>(want, rows_needed);
        const size_t rb = row_bytes(ctx);
        if (!grow_keep(ctx, ctx->keys, (size_t)want * rb, (size_t)ctx->M * rb) ||
            !grow_keep(ctx, ctx->coef, (size_t)want * 8, (size_t)ctx->M * 8))
            return fail(ctx, IQCC_ERR_OOM, "row allocation failed");
        ctx->rows_alloc = want;
        ctx->stats.rows_allocated = want;
    }
    return IQCC_OK;
}

// The key index over rows [0, M), with room for `rows_needed` entries at a
// load of at most 1/2 (the partitioned dressing and the batches look keys up
// in it; the single-Hamiltonian dress needs none).
iqcc_status ensure_index(iqcc_ctx* ctx, int64_t rows_needed) {
    const uint64_t want = pow2_at_least((uint64_t)std::max<int64_t>(rows_needed, 256) * 2);
    if (ctx->index_valid && want <= ctx->hash_slots) return IQCC_OK;
    iqcc_status st = rebuild_hash(ctx, std::max<uint64_t>(want, ctx->index_valid ? ctx->hash_slots : 0));
    if (st) return st;
    ctx->index_valid = true;
    return IQCC_OK;
}

bool bits_above_n(const iqcc_ctx* ctx, const uint64_t* w) {
    int r = ctx->n - 64 * (ctx->W - 1);
    if (r >= 64) return false;
    return (w[ctx->W - 1] >> r) != 0;
}

// Device layout of one key: x[Wd] then z[Wd].
void pad_key(const iqcc_ctx* ctx, const uint64_t* x, const uint64_t* z, uint64_t* out) {
    for (int w = 0; w < ctx->Wd; ++w) {
        out[w] = w < ctx->W ? x[w] : 0;
        out[ctx->Wd + w] = w < ctx->W ? z[w] : 0;
    }
}

SortPlan canonical_plan(const iqcc_ctx* ctx) {
    SortPlan p{};
    p.n_words = 2 * ctx->Wd;
    p.n_order = 0;
    for (int w = ctx->Wd - 1; w >= 0; --w) p.order[p.n_order++] = w;            // x, most significant first
    for (int w = ctx->Wd - 1; w >= 0; --w) p.order[p.n_order++] = ctx->Wd + w;  // then z
    return p;
}

bool is_basis(const iqcc_ctx* ctx, const double* theta) {
    for (int j = 0; j < ctx->n; ++j)
        if (!(theta[j] == 0.0 || theta[j] == kPi)) return false;
    return true;
}

void occ_words(const iqcc_ctx* ctx, const double* theta, uint64_t* occ) {
    for (int w = 0; w < 4; ++w) occ[w] = 0;
    for (int j = 0; j < ctx->n; ++j)
        if (theta[j] == kPi) occ[j / 64] |= 1ull << (j % 64);
}

int n_groups(const iqcc_ctx* ctx) { return (ctx->n + 3) / 4; }

// QMF tables for general angles, into `tables` (device), from host angles.
iqcc_status upload_tables(iqcc_ctx* ctx, const double* theta, const double* phi, double* d_angles, double* tables) {
    CK(cudaMemcpyAsync(d_angles, theta, sizeof(double) * ctx->n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(d_angles + ctx->n, phi, sizeof(double) * ctx->n, cudaMemcpyHostToDevice, ctx->stream));
    launch_qmf_tables(d_angles, d_angles + ctx->n, ctx->n, n_groups(ctx), tables, ctx->stream);
    CK_LAUNCH();
    return IQCC_OK;
}

// The other row buffer, holding at least `rows` rows (contents not kept).
iqcc_status ensure_second_rows(iqcc_ctx* ctx, int64_t rows) {
    const size_t rb = row_bytes(ctx);
    if (ctx->keys2.bytes >= (size_t)rows * rb && ctx->coef2.bytes >= (size_t)rows * 8) return IQCC_OK;
    const int64_t want = std::max<int64_t>(rows, std::min<int64_t>(ctx->capacity, ctx->rows_alloc));
    release(ctx, ctx->keys2);
    release(ctx, ctx->coef2);
    if (!ensure(ctx, ctx->keys2, (size_t)want * rb) || !ensure(ctx, ctx->coef2, (size_t)want * 8))
        return fail(ctx, IQCC_ERR_OOM, "row allocation failed");
    return IQCC_OK;
}

// The dress-bin counts ([0] = 0, then one count per bin: later their starts,
// then their ends) and the per-tile kept counts (one per tile of kDressTile
// rows and a zero: later their offsets and the total) for a dress of M rows,
// in ctx->pairbuf.
struct PairCounts {
    uint32_t* bins;
    uint32_t* tiles;
    int log2_bins;
    int64_t n_tiles;
    size_t bytes;
};

PairCounts pair_counts_layout(iqcc_ctx* ctx, int64_t M) {
    PairCounts pc;
    pc.log2_bins = pair_bins_log2(M);
    pc.n_tiles = (M + kDressTile - 1) / kDressTile;
    const size_t nb = ((size_t)1 << pc.log2_bins) + 1;
    pc.bytes = sizeof(uint32_t) * (nb + (size_t)pc.n_tiles + 1);
    pc.bins = (uint32_t*)ctx->pairbuf.p;
    pc.tiles = pc.bins ? pc.bins + nb : nullptr;
    return pc;
}

// A, B, C of padded device-layout generator pkey (all zero: energy).  With
// pair_hist the same pass counts pkey's anticommuting rows by dress bin, for
// the dress by pkey that follows (iqcc_iterate).
iqcc_status abc_impl(iqcc_ctx* ctx, const uint64_t* pkey, const double* theta, const double* phi, double* abc,
                     bool pair_hist = false) {
    const bool basis = is_basis(ctx, theta);
    uint64_t occ[4];
    occ_words(ctx, theta, occ);
    const int nb = expect_blocks();
    Carver cv;
    cv.take<double>(nb * 3);
    cv.take<double>(4);
    cv.take<double>(2 * ctx->n);
    cv.take<double>((size_t)n_groups(ctx) * 256);
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)ctx->scratch.p, 0};
    double* partials = cv.take<double>(nb * 3);
    double* out3 = cv.take<double>(4);
    double* angles = cv.take<double>(2 * ctx->n);
    double* tables = cv.take<double>((size_t)n_groups(ctx) * 256);
    if (!carve_fits(ctx, cv)) return fail(ctx, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");
    if (!basis) {
        iqcc_status st = upload_tables(ctx, theta, phi, angles, tables);
        if (st) return st;
    }
    ctx->pair_ready = false;
    PairHistOut ph{nullptr, nullptr, 0, dctr(ctx)};
    if (pair_hist && ctx->M > 0) {
        PairCounts pc = pair_counts_layout(ctx, ctx->M);
        if (!ensure(ctx, ctx->pairbuf, pc.bytes)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
        pc = pair_counts_layout(ctx, ctx->M);
        ph.log2_bins = pc.log2_bins;
        ph.counts = pc.bins + 1;
        ph.tile_kept = pc.tiles;
        CK(cudaMemsetAsync(pc.bins, 0, pc.bytes, ctx->stream));
        CK(cudaMemsetAsync(ctx->counters.p, 0, 4 * sizeof(unsigned long long), ctx->stream));
    }
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    launch_abc(ctx->Wd, ctx->rows(), ctx->c(), ctx->M, pkey, basis, occ, tables, n_groups(ctx), partials,
               ctx->stream, ph.counts ? &ph : nullptr, live_flags(ctx));
    CK_LAUNCH();
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    launch_reduce3(partials, nb, out3, ctx->stream);
    CK_LAUNCH();
    double h3[3];
    CK(cudaMemcpyAsync(h3, out3, sizeof h3, cudaMemcpyDeviceToHost, ctx->stream));
    if (ph.counts) {
        iqcc_status st = read_counters(ctx);  // synchronises the stream
        if (st) return st;
        ctx->pair_n_anti = (int64_t)ctx->h_counters->n_anti;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    ctx->stats.n_energy++;
    ctx->stats.energy_kernel_ms += ms;
    ctx->stats.energy_bytes += (double)live_terms(ctx) * (16.0 * ctx->Wd + 8.0);
    if (ph.counts) {
        ctx->pair_ready = true;
        ctx->pair_log2 = ph.log2_bins;
        std::memcpy(ctx->pair_key, pkey, sizeof(uint64_t) * 2 * ctx->Wd);
    }
    abc[0] = h3[0];
    abc[1] = h3[1];
    abc[2] = h3[2];
    return IQCC_OK;
}

iqcc_status apply_pending_cut(iqcc_ctx* ctx);

// One dress by pair partition (k_pairjoin.cu): bin histogram of the
// anticommuting rows, split (commuting rows compacted in place, anticommuting
// ones copied into their bins), join.  On IQCC_ERR_CAPACITY / OOM H is
// unchanged.  Returns the counts in *n_anti_out / *n_new_out.
// One dress by pair partition (k_pairjoin.cu), then the two row buffers swap.
// When the A, B, C pass that preceded it counted the anticommuting rows and
// the kept rows per tile (iqcc_iterate), the bins have a fixed size (the
// mean count with a quarter and 32 rows of slack): the split takes each
// row's slot in its bin and the join takes one bin per block, with no
// counting pass.  Should a bin overflow (no hash spreads that unevenly by
// chance), or without those counts, the bins are counted exactly
// (k_pair_hist), scanned, and filled and joined as contiguous ranges.  The
// split copies the commuting rows to the other row buffer at offsets known
// per tile; the join writes behind them.  On IQCC_ERR_CAPACITY / OOM H is
// unchanged.  Returns the counts in *n_anti_out / *n_new_out.
iqcc_status dress_pairs(iqcc_ctx* ctx, const PairDress& d, int64_t* n_anti_out, int64_t* n_new_out, float* ms_out) {
    const int64_t M = ctx->M;
    *n_anti_out = *n_new_out = 0;
    *ms_out = 0;
    if (M == 0) return IQCC_OK;
    // the counts of this dress were taken by the A, B, C pass that preceded it
    const bool ready = ctx->pair_ready && !d.gens && ctx->pair_log2 == pair_bins_log2(M) &&
                       std::memcmp(ctx->pair_key, d.pkey, sizeof(uint64_t) * 2 * ctx->Wd) == 0;
    ctx->pair_ready = false;
    PairCounts pc = pair_counts_layout(ctx, M);
    const uint32_t NB = 1u << pc.log2_bins;
    if (!ensure(ctx, ctx->pairbuf, pc.bytes)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    pc = pair_counts_layout(ctx, M);
    Carver cv;
    cv.take<uint32_t>(1024);
    cv.take<unsigned long long>(1);
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)ctx->scratch.p, 0};
    uint32_t* scan_tmp = cv.take<uint32_t>(1024);
    unsigned long long* out_cursor = cv.take<unsigned long long>(1);
    if (!carve_fits(ctx, cv)) return fail(ctx, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");
    DevCounters* c = dctr(ctx);
    cudaStream_t s = ctx->stream;
    CK(cudaMemsetAsync(out_cursor, 0, sizeof(unsigned long long), s));
    CK(cudaEventRecord(ctx->ev0, s));
    int64_t n_anti = 0;
    uint32_t cap = 0;  // rows per fixed-size bin; 0: exact counts
    auto count_exact = [&]() -> iqcc_status {
        CK(cudaMemsetAsync(c, 0, 4 * sizeof(unsigned long long), s));
        CK(cudaMemsetAsync(pc.bins, 0, pc.bytes, s));
        launch_pair_hist(d, ctx->rows(), M, pc.log2_bins, pc.bins + 1, pc.tiles, c, s, live_flags(ctx));
        launch_scan_u32_long(pc.bins + 1, NB, scan_tmp, s);
        launch_scan_u32_long(pc.tiles, pc.n_tiles + 1, scan_tmp, s);
        CK_LAUNCH();
        iqcc_status st2 = read_counters(ctx);
        if (st2) return st2;
        n_anti = (int64_t)ctx->h_counters->n_anti;
        cap = 0;
        return IQCC_OK;
    };
    iqcc_status st = IQCC_OK;
    if (ready) {
        n_anti = ctx->pair_n_anti;
        const double mean = (double)n_anti / (double)NB;
        const double want = std::ceil((1.0 + ctx->bin_slack) * mean) + (double)ctx->bin_slack_rows;
        if (want * (double)NB < 4.0e9 && want <= 4096.0) cap = (uint32_t)want;
        if (cap) ctx->stats.fixed_bin_dresses++;
        launch_scan_u32_long(pc.tiles, pc.n_tiles + 1, scan_tmp, s);
        CK_LAUNCH();
        if (!cap) {
            st = count_exact();
            if (st) return st;
        }
    } else {
        st = count_exact();
        if (st) return st;
    }
    *n_anti_out = n_anti;
    if (n_anti == 0) return apply_pending_cut(ctx);  // P commutes with every term
    // bin copies of the anticommuting rows: fixed-size bins when cap > 0
    const size_t slots = cap ? (size_t)NB * cap : (size_t)n_anti;
    Carver rv;
    rv.take<uint64_t>(slots * 2 * ctx->Wd);
    rv.take<double>(slots);
    if (!ensure(ctx, ctx->aux, rv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    rv = Carver{(char*)ctx->aux.p, 0};
    uint64_t* rk = rv.take<uint64_t>(slots * 2 * ctx->Wd);
    double* rc = rv.take<double>(slots);
    if (rv.off > ctx->aux.bytes) return fail(ctx, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");
    const int64_t live = live_terms(ctx);  // the rows a pending cut keeps: the input of this dress
    const uint32_t* kept = pc.tiles + pc.n_tiles;  // rows the split keeps, after the scan
    uint32_t* cursor = cap ? pc.bins : pc.bins + 1;   // fixed: per-bin counts from 0; exact: starts -> ends
    // fixed bins: up to 4 per join block, about 2048 rows and at most 4096 in all
    auto bpb_now = [&]() {
        if (!cap) return pair_bins_per_block(n_anti, pc.log2_bins);
        const double mean = (double)n_anti / (double)NB;
        uint32_t b = 1;
        while (b < 4 && 2.0 * b * mean <= 2048.0 && 2 * b * cap <= 4096) b *= 2;
        return b;
    };
    // scatter only into the bins; with fixed-size bins an overflow falls back to exact bins
    auto scatter = [&](bool compact, uint64_t* rows_out, double* coef_out) -> iqcc_status {
        if (cap) {
            CK(cudaMemsetAsync(pc.bins, 0, sizeof(uint32_t) * NB, s));
            CK(cudaMemsetAsync(&c->aux, 0, sizeof(unsigned long long), s));
        }
        launch_pair_split(d, compact, true, ctx->rows(), ctx->c(), M, pc.log2_bins, cursor, cap, rk, rc, pc.tiles,
                          rows_out, coef_out, c, s, live_flags(ctx));
        CK_LAUNCH();
        if (!cap) return IQCC_OK;
        iqcc_status st2 = read_counters(ctx);
        if (st2) return st2;
        if (ctx->h_counters->aux == 0) return IQCC_OK;
        // a bin overflowed: exact counts, contiguous bins, and the copy again
        ctx->stats.bin_overflows++;
        st2 = count_exact();
        if (st2) return st2;
        cursor = pc.bins + 1;
        launch_pair_split(d, compact, true, ctx->rows(), ctx->c(), M, pc.log2_bins, cursor, 0, rk, rc, pc.tiles,
                          rows_out, coef_out, c, s, live_flags(ctx));
        CK_LAUNCH();
        return IQCC_OK;
    };
    bool scattered = false;
    int64_t need = live + n_anti;
    if (live + n_anti > ctx->capacity) {
        // exact admission: bin copies and a counting join first, H untouched
        st = scatter(false, nullptr, nullptr);
        if (st) return st;
        launch_pair_join(d, false, rk, rc, pc.bins, pc.log2_bins, bpb_now(), nullptr, nullptr, kept, out_cursor, c, s,
                         cap);
        CK_LAUNCH();
        st = read_counters(ctx);
        if (st) return st;
        need = live + (int64_t)ctx->h_counters->n_new;
        if (need > ctx->capacity) {
            char buf[200];
            snprintf(buf, sizeof buf, "dress would need %lld rows, capacity is %lld", (long long)need,
                     (long long)ctx->capacity);
            return fail(ctx, IQCC_ERR_CAPACITY, buf);
        }
        CK(cudaMemsetAsync(&c->n_new, 0, sizeof(unsigned long long), s));
        scattered = true;
    }
    st = ensure_second_rows(ctx, std::max<int64_t>(need, 1));
    if (st) return st;
    uint64_t* rows_out = (uint64_t*)ctx->keys2.p;
    double* coef_out = (double*)ctx->coef2.p;
    if (scattered) {
        launch_pair_split(d, true, false, ctx->rows(), ctx->c(), M, pc.log2_bins, cursor, cap, rk, rc, pc.tiles,
                          rows_out, coef_out, c, s, live_flags(ctx));
        CK_LAUNCH();
    } else {
        st = scatter(true, rows_out, coef_out);
        if (st) return st;
    }
    launch_pair_join(d, true, rk, rc, pc.bins, pc.log2_bins, bpb_now(), rows_out, coef_out, kept, out_cursor, c, s,
                     cap);
    CK_LAUNCH();
    CK(cudaEventRecord(ctx->ev1, s));
    st = read_counters(ctx);
    if (st) return st;
    uint32_t mc = 0;
    unsigned long long oc = 0;
    CK(cudaMemcpyAsync(&mc, kept, sizeof mc, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&oc, out_cursor, sizeof oc, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int64_t n_new = (int64_t)ctx->h_counters->n_new;
    if ((int64_t)mc + n_anti != live || (int64_t)oc != n_anti + n_new)
        return fail(ctx, IQCC_ERR_STATE, "internal: pair dress row counts disagree");
    cudaEventElapsedTime(ms_out, ctx->ev0, ctx->ev1);
    std::swap(ctx->keys, ctx->keys2);
    std::swap(ctx->coef, ctx->coef2);
    ctx->rows_alloc = (int64_t)std::min(ctx->keys.bytes / row_bytes(ctx), ctx->coef.bytes / 8);
    ctx->stats.rows_allocated = ctx->rows_alloc;
    ctx->M = live + n_new;
    ctx->pending = false;  // the split dropped the rows of the pending cut
    ctx->index_valid = false;
    *n_new_out = n_new;
    return IQCC_OK;
}

// One generator (device-layout key); on IQCC_ERR_CAPACITY / OOM H is unchanged.
iqcc_status dress_one(iqcc_ctx* ctx, const uint64_t* pkey, double tau) {
    const int64_t M = live_terms(ctx);
    bool identity = true;
    for (int w = 0; w < 2 * ctx->Wd; ++w) identity &= pkey[w] == 0;
    if (M == 0 || identity) {
        ctx->stats.n_dress++;
        ctx->stats.dressed_terms += M;
        return apply_pending_cut(ctx);
    }
    PairDress d{ctx->Wd, pkey, nullptr, 0, std::cos(tau), std::sin(tau)};
    int64_t n_anti = 0, n_new = 0;
    float ms = 0;
    iqcc_status st = dress_pairs(ctx, d, &n_anti, &n_new, &ms);
    if (st) return st;
    iqcc_stats& s = ctx->stats;
    s.n_dress++;
    s.dressed_terms += M;
    s.anticommuting += n_anti;
    s.appended += n_new;
    s.dress_kernel_ms += ms;
    s.dress_bytes += 16.0 * ctx->Wd * (double)M + 16.0 * (double)n_anti + (16.0 * ctx->Wd + 8.0) * (double)n_new;
    return IQCC_OK;
}

// Indirect sort of rows [0, n) (or of the listed subset) in canonical order.
// Returns the sorted permutation in *out (device, inside scratch region `sc`).
struct SortArea {
    uint32_t* a;
    uint32_t* b;
    void* tmp;
    size_t tmp_bytes;
};

SortArea carve_sort(Carver& cv, int64_t n) {
    SortArea s;
    s.a = cv.take<uint32_t>(n);
    s.b = cv.take<uint32_t>(n);
    s.tmp_bytes = radix_sort_scratch_bytes(n);
    s.tmp = cv.take<char>(s.tmp_bytes);
    return s;
}

// Bytes carve_sort takes (a dry run of the same carve, so the two never differ).
size_t sort_area_bytes(int64_t n) {
    Carver dry;
    carve_sort(dry, n);
    return dry.off;
}

// rank (device [M], may be NULL): the term limit keeps the largest |rank|
// instead of the largest |C| (the magnitude threshold eps always uses |C|).
// Radix select on the bit patterns of the non-negative doubles `key` among
// the rows whose flag is set (`kept` of them), 12 bits at a time from the top
// (the first digit is the exponent), until the bucket that holds the *need-th
// largest value has at most 65,536 rows.  When the first digit is the one the
// last select chose (consecutive cuts have similar thresholds), the first pass
// also histograms the second digit of that bucket and the second pass is
// skipped.  Out: the bucket's bits (*prefix under *pmask) and, in *need, how
// many of its rows are still needed.
iqcc_status select_bucket(iqcc_ctx* ctx, const double* key, const uint8_t* flags, int64_t M, int64_t kept,
                          int64_t* need, uint64_t* prefix_out, uint64_t* pmask_out) {
    constexpr int64_t kBucketLimit = 1 << 16;
    int64_t bucket = kept;
    uint64_t prefix = 0, pmask = 0;
    int hi = 64;  // first digit: bits 52..63, the exponent (the sign bit is clear)
    if (!ensure(ctx, ctx->aux, 2 * 4096 * sizeof(unsigned long long)))
        return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    unsigned long long* hist12 = (unsigned long long*)ctx->aux.p;
    unsigned long long* hist2 = hist12 + 4096;
    std::vector<unsigned long long> h(4096), h2(4096);
    // the bucket of digit d of histogram hh holding the *need-th largest
    auto pick = [&](const std::vector<unsigned long long>& hh) {
        int64_t cum = 0;
        int sel = 0;
        for (int d = 4095; d >= 0; --d) {
            if (cum + (int64_t)hh[d] >= *need) {
                sel = d;
                break;
            }
            cum += (int64_t)hh[d];
        }
        *need -= cum;
        return sel;
    };
    bool have2 = false;  // hist2 holds the second level for the chosen first digit
    while (bucket > kBucketLimit && hi > 0) {
        const int shift = std::max(0, hi - 12);
        const bool first = hi == 64;
        CK(cudaMemsetAsync(hist12, 0, 2 * 4096 * sizeof(unsigned long long), ctx->stream));
        if (first && ctx->select_guess >= 0 && shift >= 12) {
            // one pass for two levels when the threshold's first digit is where the last select found it
            launch_abs_digit_hist12x2(key, flags, M, shift, shift - 12, (unsigned)ctx->select_guess, hist12, hist2,
                                      ctx->stream);
        } else {
            launch_abs_digit_hist12(key, flags, M, shift, prefix, pmask, hist12, ctx->stream);
        }
        CK_LAUNCH();
        CK(cudaMemcpyAsync(h.data(), hist12, 4096 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(h2.data(), hist2, 4096 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        const int sel = pick(h);
        bucket = (int64_t)h[sel];
        prefix |= (uint64_t)sel << shift;
        pmask |= (uint64_t)4095 << shift;
        hi = shift;
        if (first) {
            have2 = ctx->select_guess == sel && shift >= 12;
            ctx->select_guess = sel;
        }
        if (have2 && bucket > kBucketLimit && hi > 0) {  // the second level from the same pass
            have2 = false;
            const int shift2 = hi - 12;
            const int sel2 = pick(h2);
            bucket = (int64_t)h2[sel2];
            prefix |= (uint64_t)sel2 << shift2;
            pmask |= (uint64_t)4095 << shift2;
            hi = shift2;
        }
        have2 = false;
    }
    *prefix_out = prefix;
    *pmask_out = pmask & 0x7FFFFFFFFFFFFFFFull;
    return IQCC_OK;
}

// The rows of a term limit's threshold bucket (ties, n_cand of them, with
// `need` still to keep) kept in order of (key value desc, canonical key asc):
// their flags set.  The bucket is first ordered by the key value alone (a few
// digit passes); every row above the need-th row's value is kept, and only
// the rows that tie with that value exactly are ordered by canonical key.
iqcc_status keep_bucket_head(iqcc_ctx* ctx, const double* key, const uint32_t* ties, int64_t n_cand, int64_t need,
                             uint8_t* flags) {
    if (need >= n_cand) {
        launch_set_flags(ties, n_cand, flags, ctx->stream);
        CK_LAUNCH();
        return IQCC_OK;
    }
    if (need <= 0) return IQCC_OK;
    const int stride = 2 * ctx->Wd + 1;
    Carver dry;
    dry.take<uint64_t>((size_t)n_cand * stride);
    dry.take<uint64_t>(n_cand);
    carve_sort(dry, n_cand);
    carve_sort(dry, n_cand);
    if (!ensure(ctx, ctx->aux, dry.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    Carver cv2{(char*)ctx->aux.p, 0};
    uint64_t* skeys = cv2.take<uint64_t>((size_t)n_cand * stride);
    uint64_t* first = cv2.take<uint64_t>(n_cand);  // word 0 (the key value) in sorted order
    SortArea ca = carve_sort(cv2, n_cand);
    SortArea cb = carve_sort(cv2, n_cand);
    if (cv2.off > ctx->aux.bytes) return fail(ctx, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");
    cudaStream_t s = ctx->stream;
    launch_candidate_keys(ctx->Wd, ctx->rows(), key, ties, n_cand, skeys, s);
    launch_iota(ca.a, n_cand, s);
    SortPlan byval{};
    byval.n_words = stride;
    byval.n_order = 1;
    byval.order[0] = 0;
    uint32_t* sorted = nullptr;
    radix_sort_indirect(skeys, stride, byval, ca.a, ca.b, n_cand, &sorted, ca.tmp, ca.tmp_bytes, s);
    launch_gather_word(skeys, stride, sorted, n_cand, first, s);
    CK_LAUNCH();
    std::vector<uint64_t> h(n_cand);
    CK(cudaMemcpyAsync(h.data(), first, sizeof(uint64_t) * n_cand, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint64_t v = h[need - 1];
    int64_t lo = need - 1, hi = need;
    while (lo > 0 && h[lo - 1] == v) --lo;
    while (hi < n_cand && h[hi] == v) ++hi;
    launch_set_flags_sorted(ties, sorted, lo, flags, s);  // every row above the value
    if (hi - lo == need - lo) {
        launch_set_flags_sorted(ties, sorted + lo, hi - lo, flags, s);
    } else {  // the exact ties at the value, in canonical key order
        CK(cudaMemcpyAsync(cb.a, sorted + lo, sizeof(uint32_t) * (hi - lo), cudaMemcpyDeviceToDevice, s));
        SortPlan bykey{};
        bykey.n_words = stride;
        bykey.n_order = stride - 1;
        for (int w = 1; w < stride; ++w) bykey.order[w - 1] = w;
        uint32_t* sorted2 = nullptr;
        radix_sort_indirect(skeys, stride, bykey, cb.a, cb.b, hi - lo, &sorted2, cb.tmp, cb.tmp_bytes, s);
        launch_set_flags_sorted(ties, sorted2, need - lo, flags, s);
    }
    CK_LAUNCH();
    return IQCC_OK;
}

// Applies a pending term-limit cut: the rows it drops are compacted away.
iqcc_status apply_pending_cut(iqcc_ctx* ctx) {
    if (!ctx->pending) return IQCC_OK;
    const int64_t M = ctx->M;
    Carver cv;
    cv.take<char>(compact_inplace_scratch_bytes(M));
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    DevCounters* c = dctr(ctx);
    CK(cudaMemsetAsync(&c->aux, 0, sizeof(unsigned long long), ctx->stream));
    launch_compact_inplace(ctx->Wd, (const uint8_t*)ctx->dropflags.p, ctx->rows(), ctx->c(), M, ctx->scratch.p,
                           &c->aux, c, ctx->stream);
    CK_LAUNCH();
    iqcc_status st = read_counters(ctx);
    if (st) return st;
    ctx->M = (int64_t)ctx->h_counters->aux;
    ctx->pending = false;
    ctx->index_valid = false;
    return IQCC_OK;
}

// The term limit of App. A / Tables 2-3 (keep the max_terms largest |C|,
// ties in canonical key order) as flags only: the rows stay in place and the
// next dress drops the others while it moves rows anyway (its split), so the
// cut costs no compaction.  Only iqcc_iterate defers a cut, and only when a
// dress follows it.
iqcc_status cut_deferred(iqcc_ctx* ctx, int64_t max_terms, int64_t* removed) {
    *removed = 0;
    const int64_t M = ctx->M;
    if (ctx->pending || max_terms <= 0 || M <= max_terms) return IQCC_OK;
    ctx->pair_ready = false;
    Carver cv;
    cv.take<uint32_t>(M);  // rows of the threshold bucket
    if (!ensure(ctx, ctx->scratch, cv.off) || !ensure(ctx, ctx->dropflags, (size_t)M))
        return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    uint32_t* ties = (uint32_t*)ctx->scratch.p;
    uint8_t* flags = (uint8_t*)ctx->dropflags.p;
    DevCounters* c = dctr(ctx);
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    int64_t need = max_terms;
    uint64_t prefix = 0, pmask = 0;
    iqcc_status st = select_bucket(ctx, ctx->c(), nullptr, M, M, &need, &prefix, &pmask);
    if (st) return st;
    CK(cudaMemsetAsync(&c->aux, 0, sizeof(unsigned long long), ctx->stream));
    launch_cut_flags(ctx->c(), flags, M, prefix, pmask, ties, &c->aux, ctx->stream);
    CK_LAUNCH();
    st = read_counters(ctx);
    if (st) return st;
    st = keep_bucket_head(ctx, ctx->c(), ties, (int64_t)ctx->h_counters->aux, need, flags);
    if (st) return st;
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    ctx->stats.prune_ms += ms;
    ctx->pending = true;
    ctx->live = max_terms;
    *removed = M - max_terms;
    return IQCC_OK;
}

iqcc_status compress(iqcc_ctx* ctx, double eps, int64_t max_terms, int64_t* removed, const double* rank = nullptr) {
    ctx->pair_ready = false;
    *removed = 0;
    iqcc_status st = apply_pending_cut(ctx);
    if (st) return st;
    const int64_t M = ctx->M;
    if (M == 0) return IQCC_OK;
    const int64_t n_tiles = (M + kDressTile - 1) / kDressTile;
    Carver cv;
    cv.take<uint8_t>(M);
    cv.take<uint32_t>(n_tiles + 1);
    cv.take<uint32_t>(1024);
    cv.take<uint32_t>(M);  // tie list
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)ctx->scratch.p, 0};
    uint8_t* flags = cv.take<uint8_t>(M);
    uint32_t* tiles = cv.take<uint32_t>(n_tiles + 1);
    uint32_t* scan_tmp = cv.take<uint32_t>(1024);
    uint32_t* ties = cv.take<uint32_t>(M);
    if (!carve_fits(ctx, cv)) return fail(ctx, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");

    DevCounters* c = dctr(ctx);
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    CK(cudaMemsetAsync(c, 0, 4 * sizeof(unsigned long long), ctx->stream));
    launch_prune_flags(ctx->c(), M, eps > 0 ? eps : 0.0, flags, &c->aux, ctx->stream);
    CK_LAUNCH();
    st = read_counters(ctx);
    if (st) return st;
    const int64_t kept = (int64_t)ctx->h_counters->aux;
    if (max_terms > 0 && kept > max_terms) {
        // Radix select on the |C| bit pattern (or the rank key) down to a small
        // bucket; the bucket's rows are then ordered exactly by (|C| desc,
        // canonical key asc).
        int64_t need = max_terms;
        uint64_t prefix = 0, pmask = 0;
        st = select_bucket(ctx, rank ? rank : ctx->c(), flags, M, kept, &need, &prefix, &pmask);
        if (st) return st;
        CK(cudaMemsetAsync(&c->aux, 0, sizeof(unsigned long long), ctx->stream));
        launch_bucket_flags(rank ? rank : ctx->c(), flags, M, prefix, pmask, ties, &c->aux, ctx->stream);
        CK_LAUNCH();
        st = read_counters(ctx);
        if (st) return st;
        st = keep_bucket_head(ctx, rank ? rank : ctx->c(), ties, (int64_t)ctx->h_counters->aux, need, flags);
        if (st) return st;
    }
    // the kept rows copied into the other row buffer at offsets known per tile (no block waits on
    // another), then the buffers swap
    launch_flag_tiles(flags, M, tiles, ctx->stream);
    CK(cudaMemsetAsync(tiles + n_tiles, 0, sizeof(uint32_t), ctx->stream));
    launch_scan_u32_long(tiles, n_tiles + 1, scan_tmp, ctx->stream);
    CK_LAUNCH();
    uint32_t kept_total = 0;
    CK(cudaMemcpyAsync(&kept_total, tiles + n_tiles, sizeof kept_total, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int64_t newM = (int64_t)kept_total;
    if (newM != M) {
        st = ensure_second_rows(ctx, std::max<int64_t>(newM, 1));
        if (st) return st;
        uint64_t zero[8] = {0};
        PairDress keep{ctx->Wd, zero, nullptr, 0, 1.0, 0.0};  // no row anticommutes: the flagged rows are kept
        launch_pair_split(keep, true, false, ctx->rows(), ctx->c(), M, 10, nullptr, 0, nullptr, nullptr, tiles,
                          (uint64_t*)ctx->keys2.p, (double*)ctx->coef2.p, c, ctx->stream, flags);
        CK_LAUNCH();
    }
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    st = read_counters(ctx);
    if (st) return st;
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    ctx->stats.prune_ms += ms;
    if (newM != M) {
        std::swap(ctx->keys, ctx->keys2);
        std::swap(ctx->coef, ctx->coef2);
        ctx->rows_alloc = (int64_t)std::min(ctx->keys.bytes / row_bytes(ctx), ctx->coef.bytes / 8);
        ctx->stats.rows_allocated = ctx->rows_alloc;
        ctx->index_valid = false;  // rows moved: the index (when one is kept) is stale
    }
    ctx->M = newM;
    *removed = M - newM;
    return IQCC_OK;
}

// DIS candidates and gradients (n_cand == 0 path).  Leaves the ordered
// candidates in scratch and returns G; copies min(cap, G) to the host.
iqcc_status dis_enumerate(iqcc_ctx* ctx, const double* theta, const double* phi, int64_t cap, int64_t* n_out,
                          uint64_t* ox, uint64_t* oz, double* og) {
    const int64_t M = ctx->M;
    const int Wd = ctx->Wd, W = ctx->W;
    const bool basis = is_basis(ctx, theta);
    uint64_t occ[4];
    occ_words(ctx, theta, occ);
    // groups (distinct flip sets) are at most the rows
    const int64_t Mg = std::max<int64_t>(M, 1);
    const int nblk = expect_blocks();
    constexpr int64_t kHeadLimit = 1 << 16;  // the top-k path orders at most this many candidates
    ctx->pair_ready = false;                 // the bins below reuse the dress-bin buffer
    const int lb = pair_bins_log2(M);
    const uint32_t NB = 1u << lb;
    Carver cv;
    cv.take<uint32_t>(1024);
    cv.take<uint64_t>((size_t)Mg * Wd);
    cv.take<double>(Mg);
    cv.take<uint32_t>(kHeadLimit);
    cv.take<double>(2 * ctx->n);
    cv.take<double>((size_t)n_groups(ctx) * 256);
    cv.take<uint64_t>(16 * 2 * 4);
    cv.take<double>(std::max<size_t>((size_t)nblk * 16, 256));
    cv.take<double>(16);
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)ctx->scratch.p, 0};
    uint32_t* scan_tmp = cv.take<uint32_t>(1024);
    uint64_t* gkeys = cv.take<uint64_t>((size_t)Mg * Wd);
    double* gsum = cv.take<double>(Mg);
    uint32_t* head = cv.take<uint32_t>(kHeadLimit);
    double* angles = cv.take<double>(2 * ctx->n);
    double* tables = cv.take<double>((size_t)n_groups(ctx) * 256);
    uint64_t* cand = cv.take<uint64_t>(16 * 2 * 4);
    double* partials = cv.take<double>(std::max<size_t>((size_t)nblk * 16, 256));
    double* colsum = cv.take<double>(16);
    if (!carve_fits(ctx, cv)) return fail(ctx, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");

    DevCounters* c = dctr(ctx);
    const size_t arr_bytes = sizeof(uint32_t) * ((size_t)NB + 1);
    if (!ensure(ctx, ctx->pairbuf, arr_bytes)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    uint32_t* arr = (uint32_t*)ctx->pairbuf.p;  // [0] = 0, [1 + b]: count, then start, then end of bin b
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    // one candidate per distinct flip set: the rows grouped by flip set in a
    // partition join (k_disgroup.cu), with the z-eigenstate gradient sums
    CK(cudaMemsetAsync(c, 0, 4 * sizeof(unsigned long long), ctx->stream));
    CK(cudaMemsetAsync(arr, 0, arr_bytes, ctx->stream));
    launch_flip_hist(Wd, ctx->rows(), M, lb, arr + 1, c, ctx->stream);
    launch_scan_u32_long(arr + 1, NB, scan_tmp, ctx->stream);
    CK_LAUNCH();
    iqcc_status st = read_counters(ctx);
    if (st) return st;
    const int64_t n_flip = (int64_t)ctx->h_counters->aux;
    if (n_flip > 0) {
        if (!ensure(ctx, ctx->aux, (size_t)n_flip * flip_record_bytes(Wd)))
            return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
        launch_flip_group(Wd, ctx->rows(), ctx->c(), M, occ, basis, lb, arr, (uint64_t*)ctx->aux.p, n_flip, gkeys,
                          gsum, Mg, c, ctx->stream);
        CK_LAUNCH();
        st = read_counters(ctx);
        if (st) return st;
    }
    const int64_t G = (int64_t)ctx->h_counters->n_groups;
    if (!basis && G > 0) {
        // general angles: every term against every candidate, 16 candidates per pass
        st = upload_tables(ctx, theta, phi, angles, tables);
        if (st) return st;
        std::vector<uint64_t> hk((size_t)G * Wd);
        CK(cudaMemcpyAsync(hk.data(), gkeys, hk.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        for (int64_t g0 = 0; g0 < G; g0 += 16) {
            const int K = (int)std::min<int64_t>(16, G - g0);
            uint64_t hc[16 * 8] = {0};
            for (int k = 0; k < K; ++k) {
                bool found = false;
                for (int w = 0; w < Wd; ++w) {
                    uint64_t x = hk[(size_t)(g0 + k) * Wd + w];
                    hc[k * 2 * Wd + w] = x;
                    hc[k * 2 * Wd + Wd + w] = found ? 0 : (x & (~x + 1));
                    found |= x != 0;
                }
            }
            CK(cudaMemcpyAsync(cand, hc, sizeof(uint64_t) * 2 * Wd * K, cudaMemcpyHostToDevice, ctx->stream));
            launch_grad_general(Wd, ctx->rows(), ctx->c(), M, cand, K, tables, n_groups(ctx), partials, nblk,
                                ctx->stream);
            CK_LAUNCH();
            launch_reduce_cols(partials, nblk, 16, colsum, ctx->stream);
            CK_LAUNCH();
            CK(cudaMemcpyAsync(gsum + g0, colsum, sizeof(double) * K, cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));  // hc is reused
        }
    }
    *n_out = G;
    if (cap > 0 && G > 0) {
        SortPlan plan{};
        plan.n_words = Wd + 1;
        plan.n_order = Wd + 1;
        for (int w = 0; w <= Wd; ++w) plan.order[w] = w;
        // Order either all G candidates, or - for a short head - only those whose
        // coarse |g| reaches the cap-th largest value (radix select, 8 bits at a time).
        int64_t n_sort = G;
        bool subset = false;
        if (cap <= 64 && G > 4 * cap) {
            int64_t need = cap;
            uint64_t prefix = 0, pmask = 0;
            unsigned long long* hist = (unsigned long long*)partials;  // >= 256 words
            for (int shift = 56; shift >= 0; shift -= 8) {
                CK(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), ctx->stream));
                launch_coarse_digit_hist(gsum, G, shift, prefix, pmask, hist, ctx->stream);
                CK_LAUNCH();
                unsigned long long h[256];
                CK(cudaMemcpyAsync(h, hist, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
                CK(cudaStreamSynchronize(ctx->stream));
                int64_t cum = 0;
                int sel = 0;
                for (int d = 255; d >= 0; --d) {
                    if (cum + (int64_t)h[d] >= need) { sel = d; break; }
                    cum += (int64_t)h[d];
                }
                need -= cum;
                prefix |= (uint64_t)sel << shift;
                pmask |= (uint64_t)255 << shift;
            }
            const int64_t limit = std::min<int64_t>(G, kHeadLimit);
            CK(cudaMemsetAsync(&c->aux, 0, sizeof(unsigned long long), ctx->stream));
            launch_collect_ge(gsum, G, prefix, head, limit, &c->aux, ctx->stream);
            CK_LAUNCH();
            st = read_counters(ctx);
            if (st) return st;
            const int64_t got = (int64_t)ctx->h_counters->aux;
            if (got <= limit) {
                subset = true;
                n_sort = got;
            }
        }
        const int64_t k = std::min(cap, n_sort);
        // sort keys, permutations and the output staging, sized for this path
        Carver dry;
        dry.take<uint64_t>((size_t)n_sort * (Wd + 1));
        carve_sort(dry, n_sort);
        dry.take<uint64_t>((size_t)k * W * 2);
        dry.take<double>(k);
        if (!ensure(ctx, ctx->aux, dry.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
        Carver cv2{(char*)ctx->aux.p, 0};
        uint64_t* skeys = cv2.take<uint64_t>((size_t)n_sort * (Wd + 1));
        SortArea sa = carve_sort(cv2, n_sort);
        uint64_t* stage_x = cv2.take<uint64_t>((size_t)k * W * 2);
        double* stage_g = cv2.take<double>(k);
        if (cv2.off > ctx->aux.bytes) return fail(ctx, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");
        if (subset) launch_dis_sort_keys_sub(Wd, gkeys, gsum, head, n_sort, skeys, ctx->stream);
        else launch_dis_sort_keys(Wd, gkeys, gsum, G, skeys, ctx->stream);
        CK_LAUNCH();
        launch_iota(sa.a, n_sort, ctx->stream);
        CK_LAUNCH();
        uint32_t* sorted = nullptr;
        radix_sort_indirect(skeys, Wd + 1, plan, sa.a, sa.b, n_sort, &sorted, sa.tmp, sa.tmp_bytes, ctx->stream);
        CK_LAUNCH();
        launch_dis_export(W, Wd, gkeys, gsum, sorted, subset ? head : nullptr, k, stage_x, stage_x + (size_t)k * W,
                          stage_g, ctx->stream);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(ox, stage_x, sizeof(uint64_t) * k * W, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(oz, stage_x + (size_t)k * W, sizeof(uint64_t) * k * W, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(og, stage_g, sizeof(double) * k, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    ctx->stats.dis_ms += ms;
    return IQCC_OK;
}

iqcc_status gradients_given(iqcc_ctx* ctx, const double* theta, const double* phi, int64_t K, const uint64_t* cx,
                            const uint64_t* cz, double* grad) {
    const int Wd = ctx->Wd;
    const int nblk = expect_blocks();
    Carver cv;
    cv.take<double>(2 * ctx->n);
    cv.take<double>((size_t)n_groups(ctx) * 256);
    cv.take<uint64_t>(16 * 2 * 4);
    cv.take<double>((size_t)nblk * 16);
    cv.take<double>(16);
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)ctx->scratch.p, 0};
    double* angles = cv.take<double>(2 * ctx->n);
    double* tables = cv.take<double>((size_t)n_groups(ctx) * 256);
    uint64_t* cand = cv.take<uint64_t>(16 * 2 * 4);
    double* partials = cv.take<double>((size_t)nblk * 16);
    double* colsum = cv.take<double>(16);
    if (!carve_fits(ctx, cv)) return fail(ctx, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");
    iqcc_status st = upload_tables(ctx, theta, phi, angles, tables);
    if (st) return st;
    for (int64_t k0 = 0; k0 < K; k0 += 16) {
        const int k = (int)std::min<int64_t>(16, K - k0);
        uint64_t hc[16 * 8] = {0};
        for (int i = 0; i < k; ++i) pad_key(ctx, cx + (k0 + i) * ctx->W, cz + (k0 + i) * ctx->W, hc + i * 2 * Wd);
        CK(cudaMemcpyAsync(cand, hc, sizeof(uint64_t) * 2 * Wd * k, cudaMemcpyHostToDevice, ctx->stream));
        launch_grad_general(Wd, ctx->rows(), ctx->c(), ctx->M, cand, k, tables, n_groups(ctx), partials, nblk,
                            ctx->stream);
        CK_LAUNCH();
        launch_reduce_cols(partials, nblk, 16, colsum, ctx->stream);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(grad + k0, colsum, sizeof(double) * k, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return IQCC_OK;
}

// Union of the supports of n_gen generators (host words, W each) in device layout.
void generator_support(const iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz, uint64_t* sup) {
    for (int w = 0; w < 4; ++w) sup[w] = 0;
    for (int k = 0; k < n_gen; ++k)
        for (int w = 0; w < ctx->W; ++w) sup[w] |= gx[(size_t)k * ctx->W + w] | gz[(size_t)k * ctx->W + w];
}

// Per-qubit <sigma> (the energy-gradient table) for host angles, into scratch
// region `angles` (2n) and `tab`; returns the table's stride.
int upload_ev(iqcc_ctx* ctx, const double* theta, const double* phi, double* angles, double* tab) {
    cudaMemcpyAsync(angles, theta, sizeof(double) * ctx->n, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(angles + ctx->n, phi, sizeof(double) * ctx->n, cudaMemcpyHostToDevice, ctx->stream);
    launch_grad_tables(angles, angles + ctx->n, ctx->n, tab, ctx->stream);
    return energy_grad_table_doubles(1);
}

// Learned-screening scores of every row into `rank` (device [M]); score: optional float [M].
iqcc_status screen_scores(iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz, const double* theta,
                          const double* phi, double* rank, float* score, double* angles, double* tab) {
    if (!ctx->model.p) return fail(ctx, IQCC_ERR_ARG, "no screening model set");
    uint64_t sup[4];
    generator_support(ctx, n_gen, gx, gz, sup);
    const int ts = upload_ev(ctx, theta, phi, angles, tab);
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    launch_mlp_score(ctx->Wd, ctx->rows(), ctx->c(), ctx->M, sup, tab, ts, ctx->n, ctx->model.p, score, rank,
                     ctx->stream);
    CK_LAUNCH();
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    ctx->stats.screen_ms += ms;
    ctx->stats.screen_terms += ctx->M;
    return IQCC_OK;
}

iqcc_status prune_learned(iqcc_ctx* ctx, double eps, int64_t max_terms, int n_gen, const uint64_t* gx,
                          const uint64_t* gz, const double* theta, const double* phi, int64_t* removed) {
    *removed = 0;
    if (ctx->M == 0) return IQCC_OK;
    Buf& r = ctx->screen_rank;
    if (!ensure(ctx, r, (size_t)ctx->M * 8 + 2 * ctx->n * 8 + (size_t)energy_grad_table_doubles(ctx->n) * 8 + 1024))
        return fail(ctx, IQCC_ERR_OOM, "rank allocation failed");
    double* rank = (double*)r.p;
    double* angles = rank + ctx->M + 16;
    double* tab = angles + 2 * ctx->n + 16;
    iqcc_status st = screen_scores(ctx, n_gen, gx, gz, theta, phi, rank, nullptr, angles, tab);
    if (st) return st;
    // the magnitude floor: the floor x max_terms largest |C| (among |C| >= eps)
    // outrank every score, so the learned limit never drops them
    const int64_t M = ctx->M;
    const int64_t keep_mag = (int64_t)(ctx->screen_floor * (double)max_terms);
    if (max_terms > 0 && M > max_terms && keep_mag > 0) {
        if (!ensure(ctx, ctx->scratch, (size_t)M + (size_t)8 * (1 << 16) + 1024))
            return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
        uint8_t* flags = (uint8_t*)ctx->scratch.p;
        double* vals = (double*)((char*)ctx->scratch.p + ((M + 255) & ~(int64_t)255));
        DevCounters* c = dctr(ctx);
        CK(cudaMemsetAsync(c, 0, 4 * sizeof(unsigned long long), ctx->stream));
        launch_prune_flags(ctx->c(), M, eps > 0 ? eps : 0.0, flags, &c->aux, ctx->stream);
        CK_LAUNCH();
        st = read_counters(ctx);
        if (st) return st;
        const int64_t kept = (int64_t)ctx->h_counters->aux;
        uint64_t t_bits = 0;  // every kept row when they are no more than keep_mag
        if (kept > keep_mag) {
            int64_t need = keep_mag;
            uint64_t prefix = 0, pmask = 0;
            st = select_bucket(ctx, ctx->c(), flags, M, kept, &need, &prefix, &pmask);
            if (st) return st;
            CK(cudaMemsetAsync(&c->aux, 0, sizeof(unsigned long long), ctx->stream));
            launch_bucket_values(ctx->c(), flags, M, prefix, pmask, vals, &c->aux, 1 << 16, ctx->stream);
            CK_LAUNCH();
            st = read_counters(ctx);
            if (st) return st;
            const int64_t nb = (int64_t)ctx->h_counters->aux;
            if (nb < need) return fail(ctx, IQCC_ERR_STATE, "internal: floor bucket");
            if (nb > (1 << 16)) {
                // more than 65,536 rows left in the bucket only when all 63 bits are
                // fixed: they share one |C|, the threshold, and all of them are kept
                t_bits = prefix;
            } else {
                std::vector<uint64_t> hb((size_t)nb);
                CK(cudaMemcpyAsync(hb.data(), vals, sizeof(uint64_t) * nb, cudaMemcpyDeviceToHost, ctx->stream));
                CK(cudaStreamSynchronize(ctx->stream));
                std::nth_element(hb.begin(), hb.begin() + (need - 1), hb.end(), std::greater<uint64_t>());
                t_bits = hb[(size_t)(need - 1)];
            }
        }
        launch_boost_rank(ctx->c(), flags, M, t_bits, 1e300, rank, ctx->stream);
        CK_LAUNCH();
    }
    CK(cudaMemsetAsync(ctx->counters.p, 0, kCountersClear, ctx->stream));
    return compress(ctx, eps, max_terms, removed, rank);
}

}  // namespace

namespace iqcc {
// Message for iqcc_last_error(NULL) from entry points that have no context.
void set_thread_error(const std::string& msg) { g_last_error = msg; }
}  // namespace iqcc

// Load of packed rows in any order (k_pairjoin.cu, launch_key_group): the
// distinct keys with their coefficients summed in input order, non-zero sums
// kept, written to the row buffer in bin order; ctx->M set.  *done = false
// (nothing written) when a group of bins holds more rows than one join block
// can (many copies of one key): the caller sorts instead.
iqcc_status load_by_groups(iqcc_ctx* ctx, const uint64_t* staged, const double* c_staged, int64_t n, bool* done) {
    *done = false;
    const int L = pair_bins_log2(n);
    const uint32_t NB = 1u << L;
    const uint32_t bpb = pair_bins_per_block(n, L);
    const int Wd = ctx->Wd;
    Carver cv;
    cv.take<uint32_t>((size_t)NB + 1);
    cv.take<uint64_t>((size_t)n * 2 * Wd);
    cv.take<double>(n);
    cv.take<uint32_t>(n);
    cv.take<uint32_t>(1024);
    cv.take<unsigned long long>(1);
    if (!ensure(ctx, ctx->aux, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)ctx->aux.p, 0};
    uint32_t* counts = cv.take<uint32_t>((size_t)NB + 1);
    uint64_t* rk = cv.take<uint64_t>((size_t)n * 2 * Wd);
    double* rc = cv.take<double>(n);
    uint32_t* ri = cv.take<uint32_t>(n);
    uint32_t* scan_tmp = cv.take<uint32_t>(1024);
    unsigned long long* out_cursor = cv.take<unsigned long long>(1);
    cudaStream_t s = ctx->stream;
    DevCounters* c = dctr(ctx);
    CK(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * ((size_t)NB + 1), s));
    CK(cudaMemsetAsync(out_cursor, 0, sizeof(unsigned long long), s));
    launch_key_group(Wd, staged, c_staged, n, L, 0, counts, rk, rc, ri, bpb, nullptr, nullptr, out_cursor, c, s);
    launch_scan_u32_long(counts + 1, NB, scan_tmp, s);
    CK_LAUNCH();
    std::vector<uint32_t> h((size_t)NB + 1);
    CK(cudaMemcpyAsync(h.data(), counts + 1, sizeof(uint32_t) * NB, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h[NB] = (uint32_t)n;  // h[b]: start of bin b
    for (uint32_t g = 0; g < NB; g += bpb)
        if ((int64_t)h[std::min(g + bpb, NB)] - (int64_t)h[g] > kKeyJoinCap) return IQCC_OK;
    launch_key_group(Wd, staged, c_staged, n, L, 1, counts, rk, rc, ri, bpb, nullptr, nullptr, out_cursor, c, s);
    launch_key_group(Wd, staged, c_staged, n, L, 2, counts, rk, rc, ri, bpb, ctx->rows(), ctx->c(), out_cursor, c, s);
    CK_LAUNCH();
    iqcc_status st = read_counters(ctx);
    if (st) return st;
    unsigned long long m = 0;
    CK(cudaMemcpyAsync(&m, out_cursor, sizeof m, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->M = (int64_t)m;
    *done = true;
    return IQCC_OK;
}

extern "C" {

iqcc_status iqcc_load_hamiltonian(iqcc_ctx** out, const iqcc_opts* opts, int64_t n_terms, const uint64_t* x,
                                  const uint64_t* z, const double* coef) {
    if (!out) return fail(nullptr, IQCC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!opts) return fail(nullptr, IQCC_ERR_ARG, "opts is NULL");
    if (opts->n_qubits < 1 || opts->n_qubits > 256) return fail(nullptr, IQCC_ERR_ARG, "n_qubits must be in 1..256");
    if (n_terms < 0) return fail(nullptr, IQCC_ERR_ARG, "n_terms < 0");
    if (n_terms > 0 && (!x || !z || !coef)) return fail(nullptr, IQCC_ERR_ARG, "null input array");
    if (opts->capacity < 0 || opts->capacity > 0xFFFFFFFEll) return fail(nullptr, IQCC_ERR_ARG, "capacity out of range");
    if (opts->max_probe > kMaxProbeLimit) return fail(nullptr, IQCC_ERR_ARG, "max_probe above 256");
    if ((opts->alloc == nullptr) != (opts->free == nullptr))
        return fail(nullptr, IQCC_ERR_ARG, "alloc and free must be given together");
    iqcc_ctx* ctx = new iqcc_ctx();
    ctx->n = opts->n_qubits;
    ctx->W = (ctx->n + 63) / 64;
    ctx->Wd = device_words(ctx->n);
    ctx->capacity = opts->capacity ? opts->capacity : (int64_t)1 << 30;
    ctx->max_probe = opts->max_probe > 0 ? opts->max_probe : 64;
    ctx->stream = (cudaStream_t)opts->stream;
    ctx->device = current_device();
    ctx->alloc = opts->alloc;
    ctx->dfree = opts->free;
    ctx->alloc_user = opts->alloc_user;
    ctx->stats.words = ctx->Wd;
    auto bail = [&](iqcc_status st) {
        g_last_error = ctx->err;
        iqcc_free(ctx);
        return st;
    };
    // small inputs are checked on the host (argument errors before any device
    // work); every input is checked again on the device while it is packed
    if (n_terms <= (1 << 16))
        for (int64_t k = 0; k < n_terms; ++k)
            if (bits_above_n(ctx, x + k * ctx->W) || bits_above_n(ctx, z + k * ctx->W)) {
                fail(ctx, IQCC_ERR_ARG, "key bits set above n_qubits");
                return bail(IQCC_ERR_ARG);
            }
    if (n_terms > ctx->capacity) {
        fail(ctx, IQCC_ERR_CAPACITY, "more input terms than capacity");
        return bail(IQCC_ERR_CAPACITY);
    }
    if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->h_counters, sizeof(DevCounters)) != cudaSuccess) {
        cudaGetLastError();
        fail(ctx, IQCC_ERR_CUDA, "event / pinned allocation failed (is a CUDA device visible?)");
        return bail(IQCC_ERR_CUDA);
    }
    if (!ensure(ctx, ctx->counters, sizeof(DevCounters))) {
        fail(ctx, IQCC_ERR_OOM, "counter allocation failed");
        return bail(IQCC_ERR_OOM);
    }
    *ctx->h_counters = DevCounters{};
    ctx->h_counters->wait_limit = kDefaultWaitLimit;
    if (cudaMemcpyAsync(ctx->counters.p, ctx->h_counters, sizeof(DevCounters), cudaMemcpyHostToDevice, ctx->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        fail_cuda(ctx, cudaGetLastError(), "counter initialisation", __LINE__);
        return bail(IQCC_ERR_CUDA);
    }
    const int64_t rows0 = std::min<int64_t>(ctx->capacity, std::max<int64_t>(1024, 2 * n_terms));
    const size_t rb = row_bytes(ctx);
    if (!ensure(ctx, ctx->keys, (size_t)rows0 * rb) || !ensure(ctx, ctx->coef, (size_t)rows0 * 8)) {
        fail(ctx, IQCC_ERR_OOM, "row allocation failed");
        return bail(IQCC_ERR_OOM);
    }
    ctx->rows_alloc = rows0;
    ctx->stats.rows_allocated = rows0;
    const int64_t n = n_terms;
    if (n > 0) {
        const int W = ctx->W, Wd = ctx->Wd;
        Carver cv;
        cv.take<uint64_t>((size_t)n * W);
        cv.take<uint64_t>((size_t)n * W);
        cv.take<uint64_t>((size_t)n * 2 * Wd);  // packed rows in input order
        cv.take<double>(n);                     // coefficients in input order
        cv.take<uint8_t>(n);
        cv.take<char>(compact_inplace_scratch_bytes(n));
        cv.off += sort_area_bytes(n);
        if (!ensure(ctx, ctx->scratch, cv.off)) {
            fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
            return bail(IQCC_ERR_OOM);
        }
        cv = Carver{(char*)ctx->scratch.p, 0};
        uint64_t* dx = cv.take<uint64_t>((size_t)n * W);
        uint64_t* dz = cv.take<uint64_t>((size_t)n * W);
        uint64_t* staged = cv.take<uint64_t>((size_t)n * 2 * Wd);
        double* c_staged = cv.take<double>(n);
        uint8_t* flags = cv.take<uint8_t>(n);
        char* cscratch = cv.take<char>(compact_inplace_scratch_bytes(n));
        SortArea sa = carve_sort(cv, n);
        if (!carve_fits(ctx, cv)) {
            fail(ctx, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");
            return bail(IQCC_ERR_STATE);
        }
        cudaStream_t s = ctx->stream;
        iqcc_status st = IQCC_OK;
        do {
            if (cudaMemcpyAsync(dx, x, sizeof(uint64_t) * n * W, cudaMemcpyHostToDevice, s) ||
                cudaMemcpyAsync(dz, z, sizeof(uint64_t) * n * W, cudaMemcpyHostToDevice, s) ||
                cudaMemcpyAsync(c_staged, coef, sizeof(double) * n, cudaMemcpyHostToDevice, s)) {
                st = fail_cuda(ctx, cudaGetLastError(), "input copy", __LINE__);
                break;
            }
            // keys are checked on the device (bits above n_qubits), while packing
            const int r = ctx->n - 64 * (W - 1);
            const uint64_t hi_mask = r >= 64 ? 0ull : ~((1ull << r) - 1);
            DevCounters* cc = dctr(ctx);
            if (cudaMemsetAsync(cc, 0, 4 * sizeof(unsigned long long), s) != cudaSuccess) {
                st = fail_cuda(ctx, cudaGetLastError(), "memset", __LINE__);
                break;
            }
            launch_pack_rows(W, Wd, dx, dz, staged, n, s, hi_mask, &cc->n_new);
            launch_iota(sa.a, n, s);
            // input already in canonical order with distinct keys (an export, for one) needs no sort
            launch_order_violations(Wd, staged, n, &cc->aux, s);
            st = read_counters(ctx);
            if (st) break;
            if (ctx->h_counters->n_new != 0) {
                st = fail(ctx, IQCC_ERR_ARG, "key bits set above n_qubits");
                break;
            }
            if (ctx->h_counters->aux != 0) {
                // rows in any order: repeated keys summed by partition and join (no sort) unless a
                // group of bins is too large for one join block (many copies of one key)
                bool done = false;
                st = load_by_groups(ctx, staged, c_staged, n, &done);
                if (st) break;
                if (done) break;
            }
            uint32_t* sorted = sa.a;
            if (ctx->h_counters->aux != 0)
                radix_sort_indirect(staged, 2 * Wd, canonical_plan(ctx), sa.a, sa.b, n, &sorted, sa.tmp, sa.tmp_bytes,
                                    s);
            // run sums land in the row buffer at sorted positions; then keep the non-zero heads
            launch_sum_runs(Wd, staged, c_staged, sorted, n, flags, ctx->rows(), ctx->c(), s);
            DevCounters* c = dctr(ctx);
            launch_compact_inplace(Wd, flags, ctx->rows(), ctx->c(), n, cscratch, &c->aux, c, s);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { st = fail_cuda(ctx, e, "load kernels", __LINE__); break; }
            st = read_counters(ctx);
            if (st) break;
            ctx->M = (int64_t)ctx->h_counters->aux;
        } while (0);
        if (st) return bail(st);
    }
    ctx->index_valid = false;  // built on demand by the calls that look keys up
    ctx->launch_base = launches();
    *out = ctx;
    return IQCC_OK;
}

iqcc_status iqcc_cross_rows(iqcc_ctx* ctx, const uint64_t* gx, const uint64_t* gz, int64_t cap, int64_t* n,
                            uint64_t* x, uint64_t* z, double* coef) {
    GUARD(ctx);
    if (!gx || !gz || !n) return fail(ctx, IQCC_ERR_ARG, "null argument");
    if (cap < 0) return fail(ctx, IQCC_ERR_ARG, "cap < 0");
    if (bits_above_n(ctx, gx) || bits_above_n(ctx, gz)) return fail(ctx, IQCC_ERR_ARG, "generator bits above n_qubits");
    *n = 0;
    const int64_t M = ctx->M;
    if (M == 0) return IQCC_OK;
    const int64_t k = std::min(cap, M);
    if (k > 0 && (!x || !z || !coef)) return fail(ctx, IQCC_ERR_ARG, "null output array");
    uint64_t pk[8];
    pad_key(ctx, gx, gz, pk);
    const int W = ctx->W;
    Carver cv;
    cv.take<uint64_t>((size_t)k * W);
    cv.take<uint64_t>((size_t)k * W);
    cv.take<double>(k);
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)ctx->scratch.p, 0};
    uint64_t* dx = cv.take<uint64_t>((size_t)k * W);
    uint64_t* dz = cv.take<uint64_t>((size_t)k * W);
    double* dc = cv.take<double>(k);
    DevCounters* c = dctr(ctx);
    CK(cudaMemsetAsync(c, 0, 4 * sizeof(unsigned long long), ctx->stream));
    launch_cross_rows(ctx->Wd, ctx->rows(), ctx->c(), M, pk, W, k, dx, dz, dc, &c->aux, ctx->stream);
    CK_LAUNCH();
    iqcc_status st = read_counters(ctx);
    if (st) return st;
    *n = (int64_t)ctx->h_counters->aux;
    const int64_t out = std::min(*n, k);
    if (out > 0) {
        CK(cudaMemcpyAsync(x, dx, sizeof(uint64_t) * out * W, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(z, dz, sizeof(uint64_t) * out * W, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(coef, dc, sizeof(double) * out, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return IQCC_OK;
}

iqcc_status iqcc_dress_cross(iqcc_ctx* ctx, const uint64_t* gx, const uint64_t* gz, double tau, int64_t n_peer,
                             const uint64_t* px, const uint64_t* pz, const double* pcoef) {
    GUARD(ctx);
    if (!gx || !gz) return fail(ctx, IQCC_ERR_ARG, "null generator");
    if (n_peer < 0) return fail(ctx, IQCC_ERR_ARG, "n_peer < 0");
    if (n_peer > 0 && (!px || !pz || !pcoef)) return fail(ctx, IQCC_ERR_ARG, "null peer array");
    if (!std::isfinite(tau)) return fail(ctx, IQCC_ERR_ARG, "non-finite amplitude");
    if (bits_above_n(ctx, gx) || bits_above_n(ctx, gz)) return fail(ctx, IQCC_ERR_ARG, "generator bits above n_qubits");
    uint64_t pk[8];
    pad_key(ctx, gx, gz, pk);
    ctx->pair_ready = false;
    const int64_t M = ctx->M;
    const int64_t upper = M + n_peer;  // at most one appended row per received row
    if (upper > ctx->capacity) {
        char buf[200];
        snprintf(buf, sizeof buf, "dress would need up to %lld rows, capacity is %lld", (long long)upper,
                 (long long)ctx->capacity);
        return fail(ctx, IQCC_ERR_CAPACITY, buf);
    }
    iqcc_status st = reserve_rows(ctx, std::max<int64_t>(upper, 1));
    if (st) return st;
    st = ensure_index(ctx, std::max<int64_t>(upper, 1));
    if (st) return st;
    const int W = ctx->W, Wd = ctx->Wd;
    const uint64_t pslots = pow2_at_least((uint64_t)std::max<int64_t>(4 * n_peer, 64));  // load <= 1/4
    Carver cv;
    cv.take<uint64_t>((size_t)n_peer * W);
    cv.take<uint64_t>((size_t)n_peer * W);
    cv.take<uint64_t>((size_t)n_peer * 2 * Wd);
    cv.take<double>(n_peer);
    cv.take<uint64_t>(pslots);
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)ctx->scratch.p, 0};
    uint64_t* dx = cv.take<uint64_t>((size_t)n_peer * W);
    uint64_t* dz = cv.take<uint64_t>((size_t)n_peer * W);
    uint64_t* prow = cv.take<uint64_t>((size_t)n_peer * 2 * Wd);
    double* pc = cv.take<double>(n_peer);
    uint64_t* ps = cv.take<uint64_t>(pslots);
    DevCounters* c = dctr(ctx);
    CK(cudaMemsetAsync(c, 0, 4 * sizeof(unsigned long long), ctx->stream));
    HashView hp{ps, pslots / kBucketSlots - 1, ctx->max_probe};
    launch_hash_clear(hp, pslots, ctx->stream);  // also when no row came: every local lookup then misses
    if (n_peer > 0) {
        CK(cudaMemcpyAsync(dx, px, sizeof(uint64_t) * n_peer * W, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(dz, pz, sizeof(uint64_t) * n_peer * W, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(pc, pcoef, sizeof(double) * n_peer, cudaMemcpyHostToDevice, ctx->stream));
        const int r = ctx->n - 64 * (W - 1);
        const uint64_t hi_mask = r >= 64 ? 0ull : ~((1ull << r) - 1);
        launch_pack_rows(W, Wd, dx, dz, prow, n_peer, ctx->stream, hi_mask, &c->n_new);
        launch_hash_insert(Wd, prow, 0, n_peer, hp, c, ctx->stream);
        CK_LAUNCH();
        st = read_counters(ctx);
        if (st) return st;
        if (ctx->h_counters->n_new != 0) return fail(ctx, IQCC_ERR_ARG, "peer key bits set above n_qubits");
    }
    launch_cross_dress(Wd, ctx->rows(), ctx->c(), M, pk, std::cos(tau), std::sin(tau), hash_view(ctx), hp, prow, pc,
                       n_peer, c, ctx->stream);
    CK_LAUNCH();
    st = read_counters(ctx);
    if (st) return st;
    const int64_t n_new = (int64_t)ctx->h_counters->n_new;
    ctx->M = M + n_new;
    iqcc_stats& sx = ctx->stats;  // counted as a dress; its time is not in dress_kernel_ms
    sx.n_dress++;
    sx.dressed_terms += M;
    sx.appended += n_new;
    return IQCC_OK;
}

// One generator over two partitions a, b of one Hamiltonian on one device
// (k_pairjoin.cu, both partitions' anticommuting rows in one set of bins):
// counts of both into one bin histogram, each partition split into its own
// other row buffer and into the shared bins, one join whose outputs go to the
// partition that owns each key; then both swap their row buffers.  All work
// runs on a's stream.  On IQCC_ERR_CAPACITY / OOM both are unchanged.
static iqcc_status dress_pair_impl(iqcc_ctx* a, iqcc_ctx* b, const uint64_t* pk, double tau, const uint64_t* dmask,
                            const uint64_t* daval) {
    iqcc_ctx* ctx = a;  // CK reports on a
    cudaStream_t s = a->stream;
    iqcc_status st = apply_pending_cut(a);
    if (st) return st;
    st = apply_pending_cut(b);
    if (st) return st;
    CK(cudaStreamSynchronize(b->stream));
    a->pair_ready = b->pair_ready = false;
    const int64_t Ma = a->M, Mb = b->M;
    if (Ma + Mb == 0) return IQCC_OK;
    PairDress d{a->Wd, pk, nullptr, 0, std::cos(tau), std::sin(tau)};
    const int L = pair_bins_log2(Ma + Mb);
    const uint32_t NB = 1u << L;
    const int64_t nta = (Ma + kDressTile - 1) / kDressTile, ntb = (Mb + kDressTile - 1) / kDressTile;
    if (!ensure(a, a->pairbuf, sizeof(uint32_t) * ((size_t)NB + 1 + (size_t)nta + 1)) ||
        !ensure(b, b->pairbuf, sizeof(uint32_t) * ((size_t)ntb + 1)))
        return fail(a, IQCC_ERR_OOM, "scratch allocation failed");
    uint32_t* bins = (uint32_t*)a->pairbuf.p;
    uint32_t* ta = bins + NB + 1;
    uint32_t* tb = (uint32_t*)b->pairbuf.p;
    Carver cv;
    cv.take<uint32_t>(1024);
    cv.take<unsigned long long>(2);
    if (!ensure(a, a->scratch, cv.off)) return fail(a, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)a->scratch.p, 0};
    uint32_t* scan_tmp = cv.take<uint32_t>(1024);
    unsigned long long* cursors = cv.take<unsigned long long>(2);
    DevCounters* ca = dctr(a);
    DevCounters* cb = dctr(b);
    CK(cudaEventRecord(a->ev0, s));
    CK(cudaMemsetAsync(cursors, 0, 2 * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ca, 0, 4 * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(cb, 0, 4 * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(bins, 0, sizeof(uint32_t) * ((size_t)NB + 1 + (size_t)nta + 1), s));
    CK(cudaMemsetAsync(tb, 0, sizeof(uint32_t) * ((size_t)ntb + 1), s));
    if (Ma) launch_pair_hist(d, a->rows(), Ma, L, bins + 1, ta, ca, s);
    if (Mb) launch_pair_hist(d, b->rows(), Mb, L, bins + 1, tb, cb, s);
    launch_scan_u32_long(bins + 1, NB, scan_tmp, s);
    launch_scan_u32_long(ta, nta + 1, scan_tmp, s);
    launch_scan_u32_long(tb, ntb + 1, scan_tmp, s);
    CK_LAUNCH();
    CK(cudaStreamSynchronize(s));
    st = read_counters(a);
    if (st) return st;
    const int64_t na = (int64_t)a->h_counters->n_anti;
    st = read_counters(b);
    if (st) return st;
    const int64_t nb = (int64_t)b->h_counters->n_anti;
    const int64_t n_anti = na + nb;
    if (n_anti == 0) return IQCC_OK;
    // a partition receives at most its own anticommuting rows and one partner per row of the other
    const int64_t need_a = Ma + nb, need_b = Mb + na;
    if (need_a > a->capacity || need_b > b->capacity) {
        char buf[200];
        snprintf(buf, sizeof buf, "dress may need %lld and %lld rows, capacities are %lld and %lld",
                 (long long)need_a, (long long)need_b, (long long)a->capacity, (long long)b->capacity);
        return fail(a, IQCC_ERR_CAPACITY, buf);
    }
    Carver rv;
    rv.take<uint64_t>((size_t)n_anti * 2 * a->Wd);
    rv.take<double>(n_anti);
    if (!ensure(a, a->aux, rv.off)) return fail(a, IQCC_ERR_OOM, "scratch allocation failed");
    rv = Carver{(char*)a->aux.p, 0};
    uint64_t* rk = rv.take<uint64_t>((size_t)n_anti * 2 * a->Wd);
    double* rc = rv.take<double>(n_anti);
    st = ensure_second_rows(a, std::max<int64_t>(need_a, 1));
    if (st) return st;
    st = ensure_second_rows(b, std::max<int64_t>(need_b, 1));
    if (st) return st;
    if (Ma)
        launch_pair_split(d, true, true, a->rows(), a->c(), Ma, L, bins + 1, 0, rk, rc, ta, (uint64_t*)a->keys2.p,
                          (double*)a->coef2.p, ca, s);
    if (Mb)
        launch_pair_split(d, true, true, b->rows(), b->c(), Mb, L, bins + 1, 0, rk, rc, tb, (uint64_t*)b->keys2.p,
                          (double*)b->coef2.p, cb, s);
    PairTwo two{};
    for (int w = 0; w < 2 * a->Wd; ++w) {
        two.mask[w] = dmask[w];
        two.aval[w] = daval[w];
    }
    two.rows[0] = (uint64_t*)a->keys2.p;
    two.rows[1] = (uint64_t*)b->keys2.p;
    two.coef[0] = (double*)a->coef2.p;
    two.coef[1] = (double*)b->coef2.p;
    two.kept[0] = ta + nta;
    two.kept[1] = tb + ntb;
    two.cursor[0] = cursors;
    two.cursor[1] = cursors + 1;
    launch_pair_join2(d, rk, rc, bins, L, pair_bins_per_block(n_anti, L), two, ca, s);
    CK_LAUNCH();
    CK(cudaEventRecord(a->ev1, s));
    uint32_t kept[2] = {0, 0};
    unsigned long long got[2] = {0, 0};
    CK(cudaMemcpyAsync(&kept[0], ta + nta, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&kept[1], tb + ntb, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(got, cursors, sizeof got, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    st = read_counters(a);
    if (st) return st;
    st = read_counters(b);
    if (st) return st;
    const int64_t n_new = (int64_t)a->h_counters->n_new;
    if ((int64_t)kept[0] + na != Ma || (int64_t)kept[1] + nb != Mb ||
        (int64_t)(got[0] + got[1]) != n_anti + n_new)
        return fail(a, IQCC_ERR_STATE, "internal: two-partition dress row counts disagree");
    float ms = 0;
    cudaEventElapsedTime(&ms, a->ev0, a->ev1);
    iqcc_ctx* parts[2] = {a, b};
    const int64_t in[2] = {Ma, Mb}, anti[2] = {na, nb};
    for (int k = 0; k < 2; ++k) {
        iqcc_ctx* c = parts[k];
        std::swap(c->keys, c->keys2);
        std::swap(c->coef, c->coef2);
        c->rows_alloc = (int64_t)std::min(c->keys.bytes / row_bytes(c), c->coef.bytes / 8);
        c->stats.rows_allocated = c->rows_alloc;
        c->M = (int64_t)kept[k] + (int64_t)got[k];
        c->index_valid = false;
        c->stats.n_dress++;
        c->stats.dressed_terms += in[k];
        c->stats.anticommuting += anti[k];
        c->stats.appended += c->M - in[k];
    }
    a->stats.dress_kernel_ms += ms;
    return IQCC_OK;
}

iqcc_status iqcc_dress_pair(iqcc_ctx* a, iqcc_ctx* b, const uint64_t* gx, const uint64_t* gz, double tau,
                            const uint64_t* mx, const uint64_t* mz, const uint64_t* ax, const uint64_t* az) {
    GUARD(a);
    GUARD(b);
    if (a == b) return fail(a, IQCC_ERR_ARG, "the two partitions are one context");
    if (a->device != b->device || a->n != b->n) return fail(a, IQCC_ERR_ARG, "contexts on different devices or of different qubit counts");
    if (!gx || !gz || !mx || !mz || !ax || !az) return fail(a, IQCC_ERR_ARG, "null argument");
    if (!std::isfinite(tau)) return fail(a, IQCC_ERR_ARG, "non-finite amplitude");
    if (bits_above_n(a, gx) || bits_above_n(a, gz)) return fail(a, IQCC_ERR_ARG, "generator bits above n_qubits");
    for (int w = 0; w < a->W; ++w)
        if ((ax[w] & ~mx[w]) || (az[w] & ~mz[w])) return fail(a, IQCC_ERR_ARG, "partition bits outside the masks");
    uint64_t pk[8], dm[8], dv[8];
    pad_key(a, gx, gz, pk);
    pad_key(a, mx, mz, dm);
    pad_key(a, ax, az, dv);
    bool identity = true;
    for (int w = 0; w < 2 * a->Wd; ++w) identity &= pk[w] == 0;
    if (identity) return IQCC_OK;
    CK_CTX(a, cudaMemsetAsync(a->counters.p, 0, kCountersClear, a->stream));
    CK_CTX(b, cudaMemsetAsync(b->counters.p, 0, kCountersClear, b->stream));
    return dress_pair_impl(a, b, pk, tau, dm, dv);
}

iqcc_status iqcc_dress(iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz, const double* tau,
                       int* n_applied) {
    if (n_applied) *n_applied = 0;
    GUARD(ctx);
    if (n_gen < 0) return fail(ctx, IQCC_ERR_ARG, "n_gen < 0");
    if (n_gen > 0 && (!gx || !gz || !tau)) return fail(ctx, IQCC_ERR_ARG, "null generator array");
    for (int k = 0; k < n_gen; ++k) {
        if (bits_above_n(ctx, gx + k * ctx->W) || bits_above_n(ctx, gz + k * ctx->W))
            return fail(ctx, IQCC_ERR_ARG, "generator bits set above n_qubits");
        if (!std::isfinite(tau[k])) return fail(ctx, IQCC_ERR_ARG, "non-finite amplitude");
    }
    CK(cudaMemsetAsync(ctx->counters.p, 0, kCountersClear, ctx->stream));
    for (int k = 0; k < n_gen; ++k) {
        uint64_t pk[8];
        pad_key(ctx, gx + k * ctx->W, gz + k * ctx->W, pk);
        iqcc_status st = dress_one(ctx, pk, tau[k]);
        if (st) return st;
        if (n_applied) *n_applied = k + 1;
    }
    return IQCC_OK;
}

// One group of k generators through the sort-based path: expand every row
// along every valid path (k_sortdress.cu), sort the leaves canonically, sum
// runs of equal keys (exact zeros kept, as the hash path keeps them), compact
// into the row buffer.  The index is not touched (rebuilt by the caller).  On
// IQCC_ERR_CAPACITY / IQCC_ERR_OOM the Hamiltonian is unchanged.
iqcc_status sorted_group(iqcc_ctx* ctx, const uint64_t* pkeys, const double* tau, int k) {
    ctx->pair_ready = false;
    const int64_t M = ctx->M;
    if (M == 0) return IQCC_OK;
    const int Wd = ctx->Wd;
    DevCounters* c = dctr(ctx);
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    CK(cudaMemsetAsync(c, 0, 4 * sizeof(unsigned long long), ctx->stream));
    launch_expand_count(Wd, ctx->rows(), M, pkeys, tau, k, &c->aux, ctx->stream);
    CK_LAUNCH();
    iqcc_status st = read_counters(ctx);
    if (st) return st;
    const int64_t total = (int64_t)ctx->h_counters->aux;
    if (total > ctx->capacity) {
        char buf[200];
        snprintf(buf, sizeof buf, "sorted dress would expand to %lld rows, capacity is %lld", (long long)total,
                 (long long)ctx->capacity);
        return fail(ctx, IQCC_ERR_CAPACITY, buf);
    }
    Carver cv;
    cv.take<uint64_t>((size_t)total * 2 * Wd);
    cv.take<double>(total);
    cv.take<uint8_t>(total);
    cv.take<char>(compact_inplace_scratch_bytes(total));
    cv.off += sort_area_bytes(total);
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)ctx->scratch.p, 0};
    uint64_t* staged = cv.take<uint64_t>((size_t)total * 2 * Wd);
    double* c_staged = cv.take<double>(total);
    uint8_t* flags = cv.take<uint8_t>(total);
    char* cscratch = cv.take<char>(compact_inplace_scratch_bytes(total));
    SortArea sa = carve_sort(cv, total);
    if (!carve_fits(ctx, cv)) return fail(ctx, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");
    CK(cudaMemsetAsync(&c->aux, 0, sizeof(unsigned long long), ctx->stream));
    launch_expand_emit(Wd, ctx->rows(), ctx->c(), M, pkeys, tau, k, staged, c_staged, &c->aux, total, c, ctx->stream);
    CK_LAUNCH();
    st = read_counters(ctx);
    if (st) return st;
    if (total > ctx->rows_alloc) {  // the old rows are no longer needed: grow without keeping them
        const size_t rb = row_bytes(ctx);
        if (!ensure(ctx, ctx->keys, (size_t)total * rb) || !ensure(ctx, ctx->coef, (size_t)total * 8))
            return fail(ctx, IQCC_ERR_OOM, "row allocation failed");
        ctx->rows_alloc = total;
        ctx->stats.rows_allocated = total;
    }
    launch_iota(sa.a, total, ctx->stream);
    uint32_t* sorted = nullptr;
    radix_sort_indirect(staged, 2 * Wd, canonical_plan(ctx), sa.a, sa.b, total, &sorted, sa.tmp, sa.tmp_bytes,
                        ctx->stream);
    launch_sum_runs(Wd, staged, c_staged, sorted, total, flags, ctx->rows(), ctx->c(), ctx->stream, true);
    CK(cudaMemsetAsync(&c->aux, 0, sizeof(unsigned long long), ctx->stream));
    launch_compact_inplace(Wd, flags, ctx->rows(), ctx->c(), total, cscratch, &c->aux, c, ctx->stream);
    CK_LAUNCH();
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    st = read_counters(ctx);
    if (st) return st;
    ctx->M = (int64_t)ctx->h_counters->aux;
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    ctx->stats.sorted_dress_ms += ms;
    ctx->stats.n_sorted_groups++;
    return IQCC_OK;
}

iqcc_status iqcc_dress_sorted(iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz, const double* tau,
                              int fuse, int* n_applied) {
    if (n_applied) *n_applied = 0;
    GUARD(ctx);
    if (n_gen < 0) return fail(ctx, IQCC_ERR_ARG, "n_gen < 0");
    if (n_gen > 0 && (!gx || !gz || !tau)) return fail(ctx, IQCC_ERR_ARG, "null generator array");
    if (fuse < 1 || fuse > max_fuse()) return fail(ctx, IQCC_ERR_ARG, "fuse must be in 1..8");
    for (int k = 0; k < n_gen; ++k) {
        if (bits_above_n(ctx, gx + k * ctx->W) || bits_above_n(ctx, gz + k * ctx->W))
            return fail(ctx, IQCC_ERR_ARG, "generator bits set above n_qubits");
        if (!std::isfinite(tau[k])) return fail(ctx, IQCC_ERR_ARG, "non-finite amplitude");
    }
    CK(cudaMemsetAsync(ctx->counters.p, 0, kCountersClear, ctx->stream));
    for (int g0 = 0; g0 < n_gen; g0 += fuse) {
        const int k = std::min(fuse, n_gen - g0);
        std::vector<uint64_t> pk((size_t)k * 2 * ctx->Wd);
        for (int j = 0; j < k; ++j)
            pad_key(ctx, gx + (size_t)(g0 + j) * ctx->W, gz + (size_t)(g0 + j) * ctx->W, pk.data() + (size_t)j * 2 * ctx->Wd);
        iqcc_status st = sorted_group(ctx, pk.data(), tau + g0, k);
        if (st) return st;
        if (n_applied) *n_applied = g0 + k;
    }
    if (n_gen > 0) ctx->index_valid = false;  // rows rewritten in sorted order
    return IQCC_OK;
}

iqcc_status iqcc_prune(iqcc_ctx* ctx, double eps, int64_t max_terms, int64_t* n_removed) {
    if (n_removed) *n_removed = 0;
    GUARD(ctx);
    if (std::isnan(eps)) return fail(ctx, IQCC_ERR_ARG, "eps is NaN");
    CK(cudaMemsetAsync(ctx->counters.p, 0, kCountersClear, ctx->stream));
    int64_t removed = 0;
    iqcc_status st = compress(ctx, eps, max_terms, &removed);
    if (st) return st;
    if (n_removed) *n_removed = removed;
    return IQCC_OK;
}

// The term limit over several contexts on one device (partitions of one
// Hamiltonian): the radix select of compress() with every pass's 12-bit
// histogram summed over the parts (each part's kernel adds into one
// histogram), the threshold bucket's rows of all parts ordered together by
// (|C| desc, canonical key asc), and each part compacted with its own flags.
static iqcc_status prune_parts_impl(iqcc_ctx* const* parts, int np, double eps, int64_t max_terms, int64_t* removed) {
    iqcc_ctx* c0 = parts[0];
    cudaStream_t s0 = c0->stream;
    struct PartArea {
        uint8_t* flags;
        char* cscratch;
        uint32_t* ties;
        int64_t M, kept, n_cand;
    };
    std::vector<PartArea> pa(np);
    int64_t total = 0;
    for (int p = 0; p < np; ++p) {
        iqcc_ctx* ctx = parts[p];
        ctx->pair_ready = false;
        iqcc_status st = apply_pending_cut(ctx);
        if (st) return st;
        const int64_t M = ctx->M;
        Carver cv;
        cv.take<uint8_t>(std::max<int64_t>(M, 1));
        cv.take<char>(compact_inplace_scratch_bytes(std::max<int64_t>(M, 1)));
        cv.take<uint32_t>(std::max<int64_t>(M, 1));
        if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
        cv = Carver{(char*)ctx->scratch.p, 0};
        pa[p].flags = cv.take<uint8_t>(std::max<int64_t>(M, 1));
        pa[p].cscratch = cv.take<char>(compact_inplace_scratch_bytes(std::max<int64_t>(M, 1)));
        pa[p].ties = cv.take<uint32_t>(std::max<int64_t>(M, 1));
        pa[p].M = M;
        DevCounters* c = dctr(ctx);
        CK_CTX(ctx, cudaMemsetAsync(c, 0, 4 * sizeof(unsigned long long), ctx->stream));
        if (M > 0) {
            launch_prune_flags(ctx->c(), M, eps > 0 ? eps : 0.0, pa[p].flags, &c->aux, ctx->stream);
            CK_LAUNCH_CTX(ctx);
        }
        st = read_counters(ctx);
        if (st) return st;
        pa[p].kept = (int64_t)ctx->h_counters->aux;
        total += pa[p].kept;
    }
    if (max_terms > 0 && total > max_terms) {
        // radix select over all parts: one histogram per 12-bit pass
        constexpr int64_t kBucketLimit = 1 << 16;
        int64_t need = max_terms, bucket = total;
        uint64_t prefix = 0, pmask = 0;
        int hi = 63;
        if (!ensure(c0, c0->aux, 4096 * sizeof(unsigned long long)))
            return fail(c0, IQCC_ERR_OOM, "scratch allocation failed");
        unsigned long long* hist12 = (unsigned long long*)c0->aux.p;
        std::vector<unsigned long long> h(4096);
        while (bucket > kBucketLimit && hi > 0) {
            const int shift = std::max(0, hi - 12);
            CK_CTX(c0, cudaMemsetAsync(hist12, 0, 4096 * sizeof(unsigned long long), s0));
            CK_CTX(c0, cudaStreamSynchronize(s0));
            for (int p = 0; p < np; ++p) {
                if (pa[p].M == 0) continue;
                launch_abs_digit_hist12(parts[p]->c(), pa[p].flags, pa[p].M, shift, prefix, pmask, hist12,
                                        parts[p]->stream);
                CK_LAUNCH_CTX(parts[p]);
            }
            for (int p = 0; p < np; ++p) CK_CTX(parts[p], cudaStreamSynchronize(parts[p]->stream));
            CK_CTX(c0, cudaMemcpyAsync(h.data(), hist12, 4096 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                       s0));
            CK_CTX(c0, cudaStreamSynchronize(s0));
            int64_t cum = 0;
            int sel = 0;
            for (int d = 4095; d >= 0; --d) {
                if (cum + (int64_t)h[d] >= need) {
                    sel = d;
                    break;
                }
                cum += (int64_t)h[d];
            }
            need -= cum;
            bucket = (int64_t)h[sel];
            prefix |= (uint64_t)sel << shift;
            pmask |= (uint64_t)4095 << shift;
            hi = shift;
        }
        pmask &= 0x7FFFFFFFFFFFFFFFull;
        // the threshold bucket's rows of every part
        int64_t n_cand = 0;
        std::vector<int64_t> offs(np + 1, 0);
        for (int p = 0; p < np; ++p) {
            iqcc_ctx* ctx = parts[p];
            DevCounters* c = dctr(ctx);
            CK_CTX(ctx, cudaMemsetAsync(&c->aux, 0, sizeof(unsigned long long), ctx->stream));
            if (pa[p].M > 0) {
                launch_bucket_flags(ctx->c(), pa[p].flags, pa[p].M, prefix, pmask, pa[p].ties, &c->aux, ctx->stream);
                CK_LAUNCH_CTX(ctx);
            }
            iqcc_status st = read_counters(ctx);
            if (st) return st;
            pa[p].n_cand = (int64_t)ctx->h_counters->aux;
            offs[p] = n_cand;
            n_cand += pa[p].n_cand;
        }
        offs[np] = n_cand;
        if (need >= n_cand) {
            for (int p = 0; p < np; ++p) {
                launch_set_flags(pa[p].ties, pa[p].n_cand, pa[p].flags, parts[p]->stream);
                CK_LAUNCH_CTX(parts[p]);
            }
        } else {
            // order the candidates of all parts together, keep the first `need`
            const int stride = 2 * c0->Wd + 1;
            Carver dry;
            dry.take<uint64_t>((size_t)n_cand * stride);
            dry.take<uint32_t>(n_cand);
            dry.take<int64_t>(np + 1);
            dry.take<uint8_t*>(np);
            carve_sort(dry, n_cand);
            if (!ensure(c0, c0->aux, dry.off)) return fail(c0, IQCC_ERR_OOM, "scratch allocation failed");
            Carver cv{(char*)c0->aux.p, 0};
            uint64_t* skeys = cv.take<uint64_t>((size_t)n_cand * stride);
            uint32_t* cand = cv.take<uint32_t>(n_cand);
            int64_t* d_offs = cv.take<int64_t>(np + 1);
            uint8_t** d_flags = cv.take<uint8_t*>(np);
            SortArea ca = carve_sort(cv, n_cand);
            if (cv.off > c0->aux.bytes) return fail(c0, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");
            for (int p = 0; p < np; ++p) {
                if (pa[p].n_cand == 0) continue;
                launch_candidate_keys(c0->Wd, parts[p]->rows(), parts[p]->c(), pa[p].ties, pa[p].n_cand,
                                      skeys + (size_t)offs[p] * stride, parts[p]->stream);
                CK_LAUNCH_CTX(parts[p]);
                CK_CTX(parts[p], cudaMemcpyAsync(cand + offs[p], pa[p].ties, sizeof(uint32_t) * pa[p].n_cand,
                                                 cudaMemcpyDeviceToDevice, parts[p]->stream));
            }
            for (int p = 0; p < np; ++p) CK_CTX(parts[p], cudaStreamSynchronize(parts[p]->stream));
            std::vector<uint8_t*> hflags(np);
            for (int p = 0; p < np; ++p) hflags[p] = pa[p].flags;
            CK_CTX(c0, cudaMemcpyAsync(d_offs, offs.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice, s0));
            CK_CTX(c0, cudaMemcpyAsync(d_flags, hflags.data(), sizeof(uint8_t*) * np, cudaMemcpyHostToDevice, s0));
            launch_iota(ca.a, n_cand, s0);
            SortPlan plan{};
            plan.n_words = stride;
            plan.n_order = stride;
            for (int w = 0; w < stride; ++w) plan.order[w] = w;
            uint32_t* sorted = nullptr;
            radix_sort_indirect(skeys, stride, plan, ca.a, ca.b, n_cand, &sorted, ca.tmp, ca.tmp_bytes, s0);
            launch_set_flags_sorted_parts(cand, sorted, need, d_offs, d_flags, np, s0);
            CK_LAUNCH_CTX(c0);
            CK_CTX(c0, cudaStreamSynchronize(s0));  // the host arrays copied above live until here
        }
    }
    // each part keeps its flagged rows
    *removed = 0;
    for (int p = 0; p < np; ++p) {
        iqcc_ctx* ctx = parts[p];
        if (pa[p].M == 0) continue;
        DevCounters* c = dctr(ctx);
        CK_CTX(ctx, cudaMemsetAsync(&c->aux, 0, sizeof(unsigned long long), ctx->stream));
        launch_compact_inplace(ctx->Wd, pa[p].flags, ctx->rows(), ctx->c(), pa[p].M, pa[p].cscratch, &c->aux, c,
                               ctx->stream);
        CK_LAUNCH_CTX(ctx);
        iqcc_status st = read_counters(ctx);
        if (st) return st;
        const int64_t newM = (int64_t)ctx->h_counters->aux;
        *removed += pa[p].M - newM;
        if (newM != ctx->M) ctx->index_valid = false;
        ctx->M = newM;
    }
    return IQCC_OK;
}

iqcc_status iqcc_prune_parts(iqcc_ctx* const* parts, int n_parts, double eps, int64_t max_terms,
                             int64_t* n_removed) {
    if (n_removed) *n_removed = 0;
    if (!parts || n_parts <= 0) return fail(nullptr, IQCC_ERR_ARG, "no contexts");
    for (int p = 0; p < n_parts; ++p) {
        if (!parts[p]) return fail(nullptr, IQCC_ERR_ARG, "null context");
        if (parts[p]->broken) return IQCC_ERR_STATE;
        for (int q = 0; q < p; ++q)
            if (parts[q] == parts[p]) return fail(parts[p], IQCC_ERR_ARG, "a context is listed twice");
        if (parts[p]->device != parts[0]->device || parts[p]->n != parts[0]->n)
            return fail(parts[p], IQCC_ERR_ARG, "contexts on different devices or of different qubit counts");
    }
    if (std::isnan(eps)) return fail(parts[0], IQCC_ERR_ARG, "eps is NaN");
    for (int p = 0; p < n_parts; ++p)
        CK_CTX(parts[p], cudaMemsetAsync(parts[p]->counters.p, 0, kCountersClear, parts[p]->stream));
    int64_t removed = 0;
    iqcc_status st = prune_parts_impl(parts, n_parts, eps, max_terms, &removed);
    if (st) return st;
    if (n_removed) *n_removed = removed;
    return IQCC_OK;
}

iqcc_status iqcc_qmf_energy(iqcc_ctx* ctx, const double* theta, const double* phi, double* energy) {
    GUARD(ctx);
    if (!theta || !phi || !energy) return fail(ctx, IQCC_ERR_ARG, "null argument");
    uint64_t zero[8] = {0};
    double abc[3];
    iqcc_status st = abc_impl(ctx, zero, theta, phi, abc);
    if (st) return st;
    *energy = abc[0];
    return IQCC_OK;
}

iqcc_status iqcc_generator_abc(iqcc_ctx* ctx, const uint64_t* gx, const uint64_t* gz, const double* theta,
                               const double* phi, double abc[3]) {
    GUARD(ctx);
    if (!gx || !gz || !theta || !phi || !abc) return fail(ctx, IQCC_ERR_ARG, "null argument");
    if (bits_above_n(ctx, gx) || bits_above_n(ctx, gz)) return fail(ctx, IQCC_ERR_ARG, "generator bits above n_qubits");
    uint64_t pk[8];
    pad_key(ctx, gx, gz, pk);
    return abc_impl(ctx, pk, theta, phi, abc);
}

iqcc_status iqcc_generator_abc_parts(iqcc_ctx* const* parts, int n_parts, const uint64_t* gx, const uint64_t* gz,
                                     const double* theta, const double* phi, double abc[3], double* tau) {
    if (!parts || n_parts <= 0) return fail(nullptr, IQCC_ERR_ARG, "no contexts");
    for (int p = 0; p < n_parts; ++p) {
        GUARD(parts[p]);
        if (parts[p]->n != parts[0]->n) return fail(parts[p], IQCC_ERR_ARG, "contexts of different qubit counts");
    }
    iqcc_ctx* ctx = parts[0];
    if (!gx || !gz || !theta || !phi || !abc) return fail(ctx, IQCC_ERR_ARG, "null argument");
    if (bits_above_n(ctx, gx) || bits_above_n(ctx, gz)) return fail(ctx, IQCC_ERR_ARG, "generator bits above n_qubits");
    uint64_t pk[8];
    pad_key(ctx, gx, gz, pk);
    double sum[3] = {0.0, 0.0, 0.0};
    for (int p = 0; p < n_parts; ++p) {  // in part order: the same sum on every call
        double v[3];
        iqcc_status st = abc_impl(parts[p], pk, theta, phi, v);
        if (st) return st;
        for (int k = 0; k < 3; ++k) sum[k] += v[k];
    }
    for (int k = 0; k < 3; ++k) abc[k] = sum[k];
    if (tau) *tau = (sum[1] == 0.0 && sum[2] == 0.0) ? 0.0 : std::atan2(-sum[2], -sum[1]);
    return IQCC_OK;
}

iqcc_status iqcc_energy_gradients(iqcc_ctx* ctx, const uint64_t* gx, const uint64_t* gz, double tau,
                                  const double* theta, const double* phi, double* energy, double* d_theta,
                                  double* d_phi, double* d_tau) {
    GUARD(ctx);
    if (!theta || !phi || !energy || !d_theta || !d_phi || !d_tau) return fail(ctx, IQCC_ERR_ARG, "null argument");
    if ((gx == nullptr) != (gz == nullptr)) return fail(ctx, IQCC_ERR_ARG, "gx and gz must be given together");
    const bool has_gen = gx != nullptr;
    uint64_t pk[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (has_gen) {
        if (bits_above_n(ctx, gx) || bits_above_n(ctx, gz))
            return fail(ctx, IQCC_ERR_ARG, "generator bits above n_qubits");
        pad_key(ctx, gx, gz, pk);
    }
    const int n = ctx->n;
    const int cols = energy_grad_cols(n);
    const int nb = energy_grad_blocks();
    Carver cv;
    cv.take<double>(2 * (size_t)n);
    cv.take<double>(energy_grad_table_doubles(n));
    cv.take<double>((size_t)nb * cols);
    cv.take<double>(cols);
    cv.take<double>(2 * (size_t)n + 3);
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)ctx->scratch.p, 0};
    double* angles = cv.take<double>(2 * (size_t)n);
    double* tab = cv.take<double>(energy_grad_table_doubles(n));
    double* partials = cv.take<double>((size_t)nb * cols);
    double* sums = cv.take<double>(cols);
    double* out = cv.take<double>(2 * (size_t)n + 3);
    if (!carve_fits(ctx, cv)) return fail(ctx, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");
    std::vector<double> h(2 * (size_t)n + 3, 0.0);
    if (ctx->M > 0) {
        uint64_t occ[4];
        occ_words(ctx, theta, occ);
        CK(cudaMemcpyAsync(angles, theta, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(angles + n, phi, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
        launch_grad_tables(angles, angles + n, n, tab, ctx->stream);
        CK_LAUNCH();
        launch_energy_grad(ctx->Wd, ctx->rows(), ctx->c(), ctx->M, pk, has_gen, std::cos(tau), std::sin(tau), tab, n,
                           occ, is_basis(ctx, theta), partials, nb, ctx->stream);
        CK_LAUNCH();
        launch_reduce_cols(partials, nb, cols, sums, ctx->stream);
        CK_LAUNCH();
        launch_grad_combine(sums, tab, n, out, ctx->stream);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(h.data(), out, sizeof(double) * (2 * n + 3), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    const double A = h[2 * n], B = h[2 * n + 1], C = h[2 * n + 2];
    *energy = has_gen ? A + B * std::cos(tau) + C * std::sin(tau) : A;
    *d_tau = has_gen ? -B * std::sin(tau) + C * std::cos(tau) : 0.0;
    for (int k = 0; k < n; ++k) {
        d_theta[k] = h[k];
        d_phi[k] = h[n + k];
    }
    return IQCC_OK;
}

iqcc_status iqcc_dis_gradients(iqcc_ctx* ctx, const double* theta, const double* phi, int64_t n_cand,
                               const uint64_t* cx, const uint64_t* cz, int64_t cap, int64_t* n_out, uint64_t* ox,
                               uint64_t* oz, double* grad) {
    GUARD(ctx);
    if (!theta || !phi || !n_out) return fail(ctx, IQCC_ERR_ARG, "null argument");
    *n_out = 0;
    if (n_cand < 0 || cap < 0) return fail(ctx, IQCC_ERR_ARG, "negative count");
    if (n_cand > 0) {
        if (!cx || !cz || !grad) return fail(ctx, IQCC_ERR_ARG, "null candidate array");
        for (int64_t k = 0; k < n_cand; ++k)
            if (bits_above_n(ctx, cx + k * ctx->W) || bits_above_n(ctx, cz + k * ctx->W))
                return fail(ctx, IQCC_ERR_ARG, "candidate bits above n_qubits");
        iqcc_status st = gradients_given(ctx, theta, phi, n_cand, cx, cz, grad);
        if (st) return st;
        *n_out = n_cand;
        return IQCC_OK;
    }
    if (cap > 0 && (!ox || !oz || !grad)) return fail(ctx, IQCC_ERR_ARG, "null output array");
    CK(cudaMemsetAsync(ctx->counters.p, 0, kCountersClear, ctx->stream));
    return dis_enumerate(ctx, theta, phi, cap, n_out, ox, oz, grad);
}

iqcc_status iqcc_iterate(iqcc_ctx* ctx, const double* theta, const double* phi, const iqcc_iter_opts* o,
                         iqcc_iter_result* out) {
    GUARD(ctx);
    if (!theta || !phi || !o || !out) return fail(ctx, IQCC_ERR_ARG, "null argument");
    const int W = ctx->W;
    const int n_gen = o->n_forced > 0 ? o->n_forced : o->n_gen;
    if (n_gen < 0 || n_gen > 64) return fail(ctx, IQCC_ERR_ARG, "n_gen must be in 0..64");
    if (o->n_forced > 0 && (!o->forced_x || !o->forced_z)) return fail(ctx, IQCC_ERR_ARG, "null forced generators");
    if (o->screening != 0 && o->screening != 1) return fail(ctx, IQCC_ERR_ARG, "screening must be 0 or 1");
    if (o->screening == 1 && !ctx->model.p) return fail(ctx, IQCC_ERR_ARG, "no screening model set");
    std::memset(out, 0, sizeof *out);
    out->n_terms_before = ctx->M;
    out->n_terms_peak = ctx->M;
    const double gmin = o->min_gradient > 0 ? o->min_gradient : 1e-12;
    std::vector<uint64_t> gx((size_t)64 * W), gz((size_t)64 * W);
    std::vector<double> g(64);
    int used = 0;
    if (o->n_forced > 0) {
        used = o->n_forced;
        std::memcpy(gx.data(), o->forced_x, sizeof(uint64_t) * used * W);
        std::memcpy(gz.data(), o->forced_z, sizeof(uint64_t) * used * W);
        int64_t nn = 0;
        iqcc_status st = iqcc_dis_gradients(ctx, theta, phi, used, gx.data(), gz.data(), 0, &nn, nullptr, nullptr,
                                            g.data());
        if (st) return st;
    } else if (n_gen > 0) {
        int64_t G = 0;
        iqcc_status st = iqcc_dis_gradients(ctx, theta, phi, 0, nullptr, nullptr, n_gen, &G, gx.data(), gz.data(),
                                            g.data());
        if (st) return st;
        const int64_t avail = std::min<int64_t>(G, n_gen);
        while (used < avail && std::fabs(g[used]) > gmin) ++used;
    }
    // A term limit cut followed by another dress only marks the rows it keeps;
    // that dress drops the others as it moves rows (cut_deferred).  On an error
    // the marks are applied before returning, so H is left in one piece.
    auto fail_iter = [&](iqcc_status st) {
        if (ctx->pending && !ctx->broken) apply_pending_cut(ctx);
        return st;
    };
    for (int k = 0; k < used; ++k) {
        double abc[3];
        uint64_t pk[8];
        pad_key(ctx, gx.data() + k * W, gz.data() + k * W, pk);
        // A, B, C and the dress bins of the generator in one pass over H
        iqcc_status st = abc_impl(ctx, pk, theta, phi, abc, true);
        if (st) return fail_iter(st);
        double tau;
        if (o->n_forced > 0 && o->forced_tau) tau = o->forced_tau[k];
        else tau = (abc[1] == 0.0 && abc[2] == 0.0) ? 0.0 : std::atan2(-abc[2], -abc[1]);
        out->dressed_terms += live_terms(ctx);
        int applied = 0;
        st = iqcc_dress(ctx, 1, gx.data() + k * W, gz.data() + k * W, &tau, &applied);
        if (st) {
            out->n_applied = k;
            return fail_iter(st);
        }
        std::memcpy(out->gx + k * W, gx.data() + k * W, sizeof(uint64_t) * W);
        std::memcpy(out->gz + k * W, gz.data() + k * W, sizeof(uint64_t) * W);
        out->grad[k] = g[k];
        out->tau[k] = tau;
        for (int i = 0; i < 3; ++i) out->abc[k][i] = abc[i];
        out->n_applied = k + 1;
        out->n_terms_peak = std::max(out->n_terms_peak, ctx->M);
        if (o->max_terms > 0 && ctx->M > o->max_terms) {
            int64_t cut = 0;
            if (o->screening == 1)
                st = prune_learned(ctx, 0.0, o->max_terms, used, gx.data(), gz.data(), theta, phi, &cut);
            else if (k + 1 < used)
                st = cut_deferred(ctx, o->max_terms, &cut);
            // else: the compression below applies the same term limit (keeping the
            // max_terms largest |C| and then dropping |C| < eps keeps the same rows
            // as dropping |C| < eps and then keeping the max_terms largest)
            if (st) return fail_iter(st);
            out->n_removed += cut;
        }
    }
    int64_t removed = 0;
    iqcc_status st = o->screening == 1
                         ? prune_learned(ctx, o->eps, o->max_terms, used, gx.data(), gz.data(), theta, phi, &removed)
                         : iqcc_prune(ctx, o->eps, o->max_terms, &removed);
    if (st) return st;
    out->n_removed += removed;
    out->n_terms = ctx->M;
    return iqcc_qmf_energy(ctx, theta, phi, &out->energy);
}

iqcc_status iqcc_set_wait_limit(iqcc_ctx* ctx, int polls) {
    GUARD(ctx);
    if (polls < 0) return fail(ctx, IQCC_ERR_ARG, "polls < 0");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->h_counters->wait_limit = polls == 0 ? kDefaultWaitLimit : polls;
    CK(cudaMemcpyAsync((char*)ctx->counters.p + offsetof(DevCounters, wait_limit), &ctx->h_counters->wait_limit,
                       sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return IQCC_OK;
}

iqcc_status iqcc_set_bin_slack(iqcc_ctx* ctx, double frac, int rows) {
    GUARD(ctx);
    if (!std::isfinite(frac) || frac < 0.0 || rows < 0) return fail(ctx, IQCC_ERR_ARG, "bin slack out of range");
    ctx->bin_slack = frac;
    ctx->bin_slack_rows = rows;
    return IQCC_OK;
}

iqcc_status iqcc_wait_selftest(iqcc_ctx* ctx) {
    GUARD(ctx);
    Carver cv;
    cv.take<unsigned long long>(1);
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    unsigned long long* word = (unsigned long long*)ctx->scratch.p;
    CK(cudaMemsetAsync(ctx->counters.p, 0, kCountersClear, ctx->stream));
    CK(cudaMemsetAsync(word, 0, sizeof(unsigned long long), ctx->stream));
    launch_wait_selftest(word, dctr(ctx), ctx->stream);
    CK_LAUNCH();
    return read_counters(ctx);
}

iqcc_status iqcc_num_terms(const iqcc_ctx* ctx, int64_t* n_terms) {
    if (!ctx || !n_terms) return fail(nullptr, IQCC_ERR_ARG, "null argument");
    if (ctx->broken) return IQCC_ERR_STATE;
    *n_terms = ctx->M;
    return IQCC_OK;
}

}  // extern "C"

namespace {

// The device address of page-locked host memory registered with CUDA (it is
// mapped under unified addressing), or null for any other pointer.
void* pinned_device_view(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace

extern "C" {

iqcc_status iqcc_export_rows(iqcc_ctx* ctx, int64_t cap, int64_t* n, uint64_t* x, uint64_t* z, double* coef) {
    GUARD(ctx);
    if (!n) return fail(ctx, IQCC_ERR_ARG, "n is NULL");
    if (cap < 0) return fail(ctx, IQCC_ERR_ARG, "cap < 0");
    iqcc_status st = apply_pending_cut(ctx);
    if (st) return st;
    *n = ctx->M;
    const int64_t k = std::min(cap, ctx->M);
    if (k == 0) return IQCC_OK;
    if (!x || !z || !coef) return fail(ctx, IQCC_ERR_ARG, "null output array");
    const int W = ctx->W;
    // unpacked into device scratch, then three copies by the copy engines (faster
    // over the host link than kernel stores into mapped host memory)
    Carver cv;
    cv.take<uint64_t>((size_t)k * W);
    cv.take<uint64_t>((size_t)k * W);
    cv.take<double>(k);
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)ctx->scratch.p, 0};
    uint64_t* sx = cv.take<uint64_t>((size_t)k * W);
    uint64_t* sz = cv.take<uint64_t>((size_t)k * W);
    double* sc = cv.take<double>(k);
    launch_unpack_rows(W, ctx->Wd, ctx->rows(), ctx->c(), nullptr, sx, sz, sc, k, ctx->stream);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(x, sx, sizeof(uint64_t) * k * W, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(z, sz, sizeof(uint64_t) * k * W, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(coef, sc, sizeof(double) * k, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return IQCC_OK;
}

iqcc_status iqcc_export(iqcc_ctx* ctx, int64_t cap, int64_t* n, uint64_t* x, uint64_t* z, double* coef) {
    GUARD(ctx);
    if (!n) return fail(ctx, IQCC_ERR_ARG, "n is NULL");
    if (cap < 0) return fail(ctx, IQCC_ERR_ARG, "cap < 0");
    *n = ctx->M;
    const int64_t k = std::min(cap, ctx->M);
    if (k == 0) return IQCC_OK;
    if (!x || !z || !coef) return fail(ctx, IQCC_ERR_ARG, "null output array");
    const int64_t M = ctx->M;
    const int W = ctx->W;
    // direct radix sort of (keys, coefficient) columns, written in the export
    // layout: straight into the output arrays when they are pinned host memory
    // the device can address, else into scratch and copied
    if (!ensure(ctx, ctx->scratch, export_sort_scratch_bytes(ctx->Wd, M)))
        return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    uint64_t* dx = (uint64_t*)pinned_device_view(x);
    uint64_t* dz = (uint64_t*)pinned_device_view(z);
    double* dc = (double*)pinned_device_view(coef);
    const bool direct = dx && dz && dc;
    uint64_t* sx = nullptr;
    uint64_t* sz = nullptr;
    double* sc = nullptr;
    launch_export_sort(W, ctx->Wd, ctx->rows(), ctx->c(), M, k, ctx->scratch.p, direct ? dx : nullptr,
                       direct ? dz : nullptr, direct ? dc : nullptr, &sx, &sz, &sc, ctx->stream);
    CK_LAUNCH();
    if (!direct) {
        CK(cudaMemcpyAsync(x, sx, sizeof(uint64_t) * k * W, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(z, sz, sizeof(uint64_t) * k * W, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(coef, sc, sizeof(double) * k, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return IQCC_OK;
}

iqcc_status iqcc_set_screening_floor(iqcc_ctx* ctx, double frac) {
    GUARD(ctx);
    if (!(frac >= 0.0 && frac <= 1.0)) return fail(ctx, IQCC_ERR_ARG, "floor must be in [0, 1]");
    ctx->screen_floor = frac;
    return IQCC_OK;
}

iqcc_status iqcc_set_screening_model(iqcc_ctx* ctx, const float* w1, const float* b1, const float* w2,
                                     const float* b2, const float* w3, float b3) {
    GUARD(ctx);
    if (!w1 || !b1 || !w2 || !b2 || !w3) return fail(ctx, IQCC_ERR_ARG, "null weight array");
    std::vector<unsigned char> h(screen_model_bytes());
    pack_screen_model(w1, b1, w2, b2, w3, b3, h.data());
    if (!ensure(ctx, ctx->model, h.size())) return fail(ctx, IQCC_ERR_OOM, "model allocation failed");
    CK(cudaMemcpyAsync(ctx->model.p, h.data(), h.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return IQCC_OK;
}

}  // extern "C"

namespace {

// Canonical (export) order of the rows into perm (device [M]) through the sort area.
iqcc_status canonical_order(iqcc_ctx* ctx, const SortArea& sa, uint32_t** perm) {
    launch_iota(sa.a, ctx->M, ctx->stream);
    radix_sort_indirect(ctx->rows(), 2 * ctx->Wd, canonical_plan(ctx), sa.a, sa.b, ctx->M, perm, sa.tmp,
                        sa.tmp_bytes, ctx->stream);
    CK_LAUNCH();
    return IQCC_OK;
}

// One per-row quantity of the screening family, in export order, to the host:
// kind 0 features (float [M][8]), 1 future energies (double [M]), 2 scores (float [M]).
iqcc_status per_row_export(iqcc_ctx* ctx, int kind, int n_gen, const uint64_t* gx, const uint64_t* gz,
                           const double* tau, const double* theta, const double* phi, void* out) {
    const int64_t M = ctx->M;
    if (M == 0) return IQCC_OK;
    const int n = ctx->n;
    const size_t width = kind == 0 ? (size_t)screen_features() * 4 : (kind == 1 ? 8 : 4);
    Carver cv;
    cv.off += sort_area_bytes(M);
    cv.take<char>((size_t)M * width);
    cv.take<char>((size_t)M * width);
    cv.take<double>(M);
    cv.take<double>(2 * (size_t)n);
    cv.take<double>(energy_grad_table_doubles(n));
    if (!ensure(ctx, ctx->scratch, cv.off)) return fail(ctx, IQCC_ERR_OOM, "scratch allocation failed");
    cv = Carver{(char*)ctx->scratch.p, 0};
    SortArea sa = carve_sort(cv, M);
    char* vals = cv.take<char>((size_t)M * width);
    char* sorted_vals = cv.take<char>((size_t)M * width);
    double* rank = cv.take<double>(M);
    double* angles = cv.take<double>(2 * (size_t)n);
    double* tab = cv.take<double>(energy_grad_table_doubles(n));
    if (!carve_fits(ctx, cv)) return fail(ctx, IQCC_ERR_STATE, "internal: scratch carve exceeds allocation");
    uint64_t sup[4];
    generator_support(ctx, n_gen, gx, gz, sup);
    if (kind == 0) {
        const int ts = upload_ev(ctx, theta, phi, angles, tab);
        launch_term_features(ctx->Wd, ctx->rows(), ctx->c(), M, sup, tab, ts, n, (float*)vals, ctx->stream);
    } else if (kind == 1) {
        const int ts = upload_ev(ctx, theta, phi, angles, tab);
        std::vector<uint64_t> pk((size_t)std::max(n_gen, 1) * 2 * ctx->Wd);
        for (int j = 0; j < n_gen; ++j)
            pad_key(ctx, gx + (size_t)j * ctx->W, gz + (size_t)j * ctx->W, pk.data() + (size_t)j * 2 * ctx->Wd);
        launch_future_energy(ctx->Wd, ctx->rows(), M, pk.data(), tau, n_gen, tab, ts, n, (double*)vals, ctx->stream);
    } else {
        iqcc_status st = screen_scores(ctx, n_gen, gx, gz, theta, phi, rank, (float*)vals, angles, tab);
        if (st) return st;
    }
    CK_LAUNCH();
    uint32_t* perm = nullptr;
    iqcc_status st = canonical_order(ctx, sa, &perm);
    if (st) return st;
    launch_gather_bytes(vals, perm, M, (int)width, sorted_vals, ctx->stream);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(out, sorted_vals, (size_t)M * width, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return IQCC_OK;
}

iqcc_status check_gens(iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz, int max_gen) {
    if (n_gen < 0 || n_gen > max_gen) return fail(ctx, IQCC_ERR_ARG, "generator count out of range");
    if (n_gen > 0 && (!gx || !gz)) return fail(ctx, IQCC_ERR_ARG, "null generator array");
    for (int k = 0; k < n_gen; ++k)
        if (bits_above_n(ctx, gx + (size_t)k * ctx->W) || bits_above_n(ctx, gz + (size_t)k * ctx->W))
            return fail(ctx, IQCC_ERR_ARG, "generator bits set above n_qubits");
    return IQCC_OK;
}

}  // namespace

extern "C" {

iqcc_status iqcc_term_features(iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz, const double* theta,
                               const double* phi, float* out) {
    GUARD(ctx);
    if (!theta || !phi || (ctx->M > 0 && !out)) return fail(ctx, IQCC_ERR_ARG, "null argument");
    iqcc_status st = check_gens(ctx, n_gen, gx, gz, 64);
    if (st) return st;
    return per_row_export(ctx, 0, n_gen, gx, gz, nullptr, theta, phi, out);
}

iqcc_status iqcc_future_energies(iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz, const double* tau,
                                 const double* theta, const double* phi, double* out) {
    GUARD(ctx);
    if (!theta || !phi || (n_gen > 0 && !tau) || (ctx->M > 0 && !out)) return fail(ctx, IQCC_ERR_ARG, "null argument");
    iqcc_status st = check_gens(ctx, n_gen, gx, gz, max_fuse());
    if (st) return st;
    for (int k = 0; k < n_gen; ++k)
        if (!std::isfinite(tau[k])) return fail(ctx, IQCC_ERR_ARG, "non-finite amplitude");
    return per_row_export(ctx, 1, n_gen, gx, gz, tau, theta, phi, out);
}

iqcc_status iqcc_term_scores(iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz, const double* theta,
                             const double* phi, float* out) {
    GUARD(ctx);
    if (!theta || !phi || (ctx->M > 0 && !out)) return fail(ctx, IQCC_ERR_ARG, "null argument");
    iqcc_status st = check_gens(ctx, n_gen, gx, gz, 64);
    if (st) return st;
    return per_row_export(ctx, 2, n_gen, gx, gz, nullptr, theta, phi, out);
}

iqcc_status iqcc_prune_learned(iqcc_ctx* ctx, double eps, int64_t max_terms, int n_gen, const uint64_t* gx,
                               const uint64_t* gz, const double* theta, const double* phi, int64_t* n_removed) {
    if (n_removed) *n_removed = 0;
    GUARD(ctx);
    if (std::isnan(eps) || !theta || !phi) return fail(ctx, IQCC_ERR_ARG, "bad argument");
    iqcc_status st = check_gens(ctx, n_gen, gx, gz, 64);
    if (st) return st;
    int64_t removed = 0;
    st = prune_learned(ctx, eps, max_terms, n_gen, gx, gz, theta, phi, &removed);
    if (st) return st;
    if (n_removed) *n_removed = removed;
    return IQCC_OK;
}

iqcc_status iqcc_get_stats(const iqcc_ctx* ctx, iqcc_stats* out) {
    if (!ctx || !out) return fail(nullptr, IQCC_ERR_ARG, "null argument");
    *out = ctx->stats;
    out->kernel_launches = launches() - ctx->launch_base;
    return IQCC_OK;
}

iqcc_status iqcc_reset_stats(iqcc_ctx* ctx) {
    if (!ctx) return fail(nullptr, IQCC_ERR_ARG, "null context");
    iqcc_stats s{};
    s.rows_allocated = ctx->rows_alloc;
    s.hash_slots = (int64_t)ctx->hash_slots;
    s.words = ctx->Wd;
    ctx->stats = s;
    ctx->launch_base = launches();
    return IQCC_OK;
}

const char* iqcc_last_error(const iqcc_ctx* ctx) {
    if (!ctx) return g_last_error.c_str();
    return ctx->err.empty() ? "no error" : ctx->err.c_str();
}

void iqcc_free(iqcc_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    release(ctx, ctx->keys);
    release(ctx, ctx->coef);
    release(ctx, ctx->hash);
    release(ctx, ctx->counters);
    release(ctx, ctx->scratch);
    release(ctx, ctx->aux);
    release(ctx, ctx->model);
    release(ctx, ctx->screen_rank);
    release(ctx, ctx->pairbuf);
    release(ctx, ctx->keys2);
    release(ctx, ctx->coef2);
    release(ctx, ctx->dropflags);
    if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    cudaGetLastError();
    delete ctx;
}

}  // extern "C"

// ============================================================================
// Batches of independent Hamiltonians
// ============================================================================

struct iqcc_batch {
    iqcc_ctx* ctx = nullptr;
    int B = 0;
    std::vector<int> n;          // qubits per problem
    std::vector<int64_t> aoff;   // offsets into the concatenated angle arrays
    Buf dev;                     // per-problem device arrays (carved)
    Buf groups;                  // DIS group slots and sums
    uint64_t group_slots = 0;
    cudaStream_t gs = nullptr;   // stream the screening graph runs on
    cudaGraphExec_t graph = nullptr;
    int64_t graph_M = -1;
    uint64_t* h_occ = nullptr;   // pinned [B]
    char* h_out = nullptr;       // pinned results
    int blocks[3] = {0, 0, 0};   // tuned grids: energy, group, abc
    int64_t screens = 0, replays = 0;
};

namespace {

constexpr uint64_t kBatchXMask = (1ull << kBatchTagShift) - 1;

// Device arrays of a batch, carved from b->dev.
struct BatchDev {
    uint64_t* occ;
    unsigned long long* best_coarse;
    unsigned long long* best_key;
    double* best_g;
    double* energy;
    double* abc;
    double* tau;
    unsigned long long* counts;
    Gen<1>* gens;
    double* part_e;
    double* part_abc;
};

int batch_max_blocks() { return sm_count() * 16; }

BatchDev carve_batch(Carver& cv, int B) {
    BatchDev d;
    d.occ = cv.take<uint64_t>(B);
    d.best_coarse = cv.take<unsigned long long>(B);
    d.best_key = cv.take<unsigned long long>(B);
    d.best_g = cv.take<double>(B);
    d.energy = cv.take<double>(B);
    d.abc = cv.take<double>(3 * (size_t)B);
    d.tau = cv.take<double>(B);
    d.counts = cv.take<unsigned long long>(B);
    d.gens = cv.take<Gen<1>>(B);
    d.part_e = cv.take<double>((size_t)batch_max_blocks() * B);
    d.part_abc = cv.take<double>((size_t)batch_max_blocks() * 3 * B);
    return d;
}

// Pinned result block: energy, best_key, best_g, abc, tau, counts.
size_t batch_out_bytes(int B) { return (size_t)B * (8 + 8 + 8 + 24 + 8 + 8); }

// The screening sequence on b->gs (no host synchronisation inside).
void enqueue_screen(iqcc_batch* b, const BatchDev& d, const int* blocks) {
    iqcc_ctx* ctx = b->ctx;
    const int B = b->B;
    cudaStream_t s = b->gs;
    cudaMemcpyAsync(d.occ, b->h_occ, sizeof(uint64_t) * B, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(d.counts, 0, sizeof(unsigned long long) * B, s);
    cudaMemsetAsync(d.best_coarse, 0, sizeof(unsigned long long) * B, s);
    cudaMemsetAsync(d.best_key, 0xFF, sizeof(unsigned long long) * B, s);
    cudaMemsetAsync(d.best_g, 0, sizeof(double) * B, s);
    uint64_t* slots = (uint64_t*)b->groups.p;
    double* gsum = (double*)(slots + b->group_slots);
    cudaMemsetAsync(slots, 0xFF, sizeof(uint64_t) * b->group_slots, s);
    cudaMemsetAsync(gsum, 0, sizeof(double) * b->group_slots, s);
    launch_seg_energy(ctx->rows(), ctx->c(), ctx->M, d.occ, B, d.part_e, d.counts, blocks[0], s);
    launch_reduce_cols(d.part_e, blocks[0], B, d.energy, s);
    launch_seg_dis_group(ctx->rows(), ctx->c(), ctx->M, d.occ, B, slots, gsum, b->group_slots / kBucketSlots - 1,
                         ctx->max_probe, dctr(ctx), blocks[1], s);
    launch_seg_best(slots, gsum, b->group_slots, B, d.best_coarse, d.best_key, d.best_g, blocks[1], s);
    launch_seg_abc(ctx->rows(), ctx->c(), ctx->M, d.occ, B, d.best_key, d.part_abc, blocks[2], s);
    launch_reduce_cols(d.part_abc, blocks[2], 3 * B, d.abc, s);
    launch_seg_tau(d.abc, d.best_key, B, d.tau, d.gens, s);
    char* o = b->h_out;
    cudaMemcpyAsync(o, d.energy, sizeof(double) * B, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(o + 8 * B, d.best_key, sizeof(uint64_t) * B, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(o + 16 * B, d.best_g, sizeof(double) * B, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(o + 24 * B, d.abc, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(o + 48 * B, d.tau, sizeof(double) * B, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(o + 56 * B, d.counts, sizeof(uint64_t) * B, cudaMemcpyDeviceToHost, s);
}

// Launch shapes by measurement: each screening kernel at 2, 4, 8 and 16 blocks
// per SM, the fastest kept (one untimed run first fills the candidate arrays).
iqcc_status tune_batch(iqcc_batch* b, const BatchDev& d) {
    iqcc_ctx* ctx = b->ctx;
    const int B = b->B;
    const int sm = sm_count();
    int blocks[3] = {4 * sm, 4 * sm, 4 * sm};
    enqueue_screen(b, d, blocks);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    uint64_t* slots = (uint64_t*)b->groups.p;
    double* gsum = (double*)(slots + b->group_slots);
    float best[3] = {1e30f, 1e30f, 1e30f};
    for (int mult : {2, 4, 8, 16}) {
        const int g = mult * sm;
        float ms[3] = {0, 0, 0};
        for (int k = 0; k < 3; ++k) {
            if (k == 1) {
                cudaMemsetAsync(slots, 0xFF, sizeof(uint64_t) * b->group_slots, b->gs);
                cudaMemsetAsync(gsum, 0, sizeof(double) * b->group_slots, b->gs);
            }
            cudaEventRecord(e0, b->gs);
            if (k == 0) launch_seg_energy(ctx->rows(), ctx->c(), ctx->M, d.occ, B, d.part_e, d.counts, g, b->gs);
            if (k == 1)
                launch_seg_dis_group(ctx->rows(), ctx->c(), ctx->M, d.occ, B, slots, gsum,
                                     b->group_slots / kBucketSlots - 1, ctx->max_probe, dctr(ctx), g, b->gs);
            if (k == 2) launch_seg_abc(ctx->rows(), ctx->c(), ctx->M, d.occ, B, d.best_key, d.part_abc, g, b->gs);
            cudaEventRecord(e1, b->gs);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms[k], e0, e1);
            if (ms[k] < best[k]) {
                best[k] = ms[k];
                b->blocks[k] = g;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaStreamSynchronize(b->gs));
    return IQCC_OK;
}

// capture: on a state without a valid graph, capture one (else run the sequence directly).
iqcc_status batch_screen(iqcc_batch* b, const double* theta, const double* phi, iqcc_batch_screen_out* out,
                         bool capture) {
    iqcc_ctx* ctx = b->ctx;
    const int B = b->B;
    if (!theta || !phi || !out || !out->energy || !out->gx || !out->gz || !out->grad || !out->abc || !out->tau ||
        !out->n_terms)
        return fail(ctx, IQCC_ERR_ARG, "null argument");
    for (int p = 0; p < B; ++p) {
        uint64_t occ = 0;
        for (int j = 0; j < b->n[p]; ++j) {
            const double t = theta[b->aoff[p] + j];
            if (!(t == 0.0 || t == kPi)) return fail(ctx, IQCC_ERR_ARG, "batched screening needs theta 0 or pi");
            if (t == kPi) occ |= 1ull << j;
        }
        b->h_occ[p] = occ;
    }
    // group table for at most one group per term, load <= 1/2
    const uint64_t want = pow2_at_least((uint64_t)std::max<int64_t>(ctx->M, 256) * 2);
    if (want != b->group_slots) {
        if (!ensure(ctx, b->groups, (size_t)want * 16)) return fail(ctx, IQCC_ERR_OOM, "group table allocation failed");
        b->group_slots = want;
        b->graph_M = -1;
    }
    Carver cv{(char*)b->dev.p, 0};
    const BatchDev d = carve_batch(cv, B);
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemsetAsync(ctx->counters.p, 0, kCountersClear, b->gs));
    if (b->graph && b->graph_M == ctx->M) {
        CK(cudaGraphLaunch(b->graph, b->gs));
        b->replays++;
    } else {
        if (!b->blocks[0]) {
            iqcc_status st = tune_batch(b, d);
            if (st) return st;
        }
        if (!capture) {
            enqueue_screen(b, d, b->blocks);
            CK_LAUNCH();
        } else {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(b->gs, cudaStreamCaptureModeThreadLocal));
        enqueue_screen(b, d, b->blocks);
        CK(cudaStreamEndCapture(b->gs, &g));
        const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        b->graph_M = ctx->M;
        CK(cudaGraphLaunch(b->graph, b->gs));
        }
    }
    CK(cudaStreamSynchronize(b->gs));
    b->screens++;
    CK(cudaMemcpy(ctx->h_counters, ctx->counters.p, sizeof(DevCounters), cudaMemcpyDeviceToHost));
    if (ctx->h_counters->err) {
        char buf[160];
        snprintf(buf, sizeof buf, "device error %d raised by kernel site %d", ctx->h_counters->err,
                 ctx->h_counters->err_where);
        return fail(ctx, (iqcc_status)ctx->h_counters->err, buf);
    }
    const char* o = b->h_out;
    for (int p = 0; p < B; ++p) {
        const uint64_t key = ((const uint64_t*)(o + 8 * B))[p];
        const bool none = key == kEmptySlot;
        out->energy[p] = ((const double*)o)[p];
        out->gx[p] = none ? 0 : (key & kBatchXMask);
        out->gz[p] = out->gx[p] & (~out->gx[p] + 1);
        out->grad[p] = ((const double*)(o + 16 * B))[p];
        for (int k = 0; k < 3; ++k) out->abc[3 * p + k] = ((const double*)(o + 24 * B))[3 * p + k];
        out->tau[p] = ((const double*)(o + 48 * B))[p];
        out->n_terms[p] = (int64_t)((const uint64_t*)(o + 56 * B))[p];
    }
    return IQCC_OK;
}

}  // namespace

extern "C" {

iqcc_status iqcc_batch_load(iqcc_batch** out, const iqcc_opts* opts, int n_problems, const int* n_qubits,
                            const int64_t* offsets, const uint64_t* x, const uint64_t* z, const double* coef) {
    if (!out) return fail(nullptr, IQCC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!opts || !n_qubits || !offsets) return fail(nullptr, IQCC_ERR_ARG, "null argument");
    if (n_problems < 1 || n_problems > kMaxBatch) return fail(nullptr, IQCC_ERR_ARG, "n_problems must be in 1..2048");
    if (offsets[0] != 0) return fail(nullptr, IQCC_ERR_ARG, "offsets[0] must be 0");
    const int B = n_problems;
    for (int b = 0; b < B; ++b) {
        if (n_qubits[b] < 1 || n_qubits[b] > kBatchTagShift)
            return fail(nullptr, IQCC_ERR_ARG, "problem qubit counts must be in 1..48");
        if (offsets[b + 1] < offsets[b]) return fail(nullptr, IQCC_ERR_ARG, "offsets must not decrease");
    }
    const int64_t M = offsets[B];
    if (M > 0 && (!x || !z || !coef)) return fail(nullptr, IQCC_ERR_ARG, "null input array");
    std::vector<uint64_t> zt((size_t)M);
    for (int b = 0; b < B; ++b) {
        const uint64_t hi = n_qubits[b] >= 64 ? 0ull : ~((1ull << n_qubits[b]) - 1);
        for (int64_t i = offsets[b]; i < offsets[b + 1]; ++i) {
            if ((x[i] | z[i]) & hi) return fail(nullptr, IQCC_ERR_ARG, "key bits set above a problem's qubit count");
            zt[i] = z[i] | ((uint64_t)b << kBatchTagShift);
        }
    }
    iqcc_opts o = *opts;
    o.n_qubits = 64;
    iqcc_ctx* ctx = nullptr;
    iqcc_status st = iqcc_load_hamiltonian(&ctx, &o, M, x, zt.data(), coef);
    if (st) return st;
    iqcc_batch* b = new iqcc_batch();
    b->ctx = ctx;
    b->B = B;
    b->n.assign(n_qubits, n_qubits + B);
    b->aoff.resize(B + 1, 0);
    for (int p = 0; p < B; ++p) b->aoff[p + 1] = b->aoff[p] + n_qubits[p];
    Carver dry;
    carve_batch(dry, B);
    bool ok = cudaStreamCreateWithFlags(&b->gs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMallocHost((void**)&b->h_occ, sizeof(uint64_t) * B) == cudaSuccess &&
              cudaMallocHost((void**)&b->h_out, batch_out_bytes(B)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        set_thread_error("batch stream / pinned allocation failed");
        iqcc_batch_free(b);
        return IQCC_ERR_CUDA;
    }
    if (!ensure(ctx, b->dev, dry.off)) {
        set_thread_error("batch allocation failed");
        iqcc_batch_free(b);
        return IQCC_ERR_OOM;
    }
    *out = b;
    return IQCC_OK;
}

iqcc_status iqcc_batch_screen(iqcc_batch* b, const double* theta, const double* phi, iqcc_batch_screen_out* out) {
    if (!b) return fail(nullptr, IQCC_ERR_ARG, "null batch");
    GUARD(b->ctx);
    return batch_screen(b, theta, phi, out, true);
}

iqcc_status iqcc_batch_step(iqcc_batch* b, const double* theta, const double* phi, double eps,
                            iqcc_batch_screen_out* out, double* energy_after, int64_t* n_terms_after) {
    if (!b) return fail(nullptr, IQCC_ERR_ARG, "null batch");
    iqcc_ctx* ctx = b->ctx;
    GUARD(ctx);
    if (std::isnan(eps)) return fail(ctx, IQCC_ERR_ARG, "eps is NaN");
    if (2 * ctx->M > ctx->capacity)
        return fail(ctx, IQCC_ERR_CAPACITY, "a batch step needs capacity for twice the current terms");
    iqcc_status st = batch_screen(b, theta, phi, out, false);
    if (st) return st;
    Carver cv{(char*)b->dev.p, 0};
    const BatchDev d = carve_batch(cv, b->B);
    const int64_t M = ctx->M;
    if (M > 0) {
        // each row dressed by its problem's generator, by pair partition
        PairDress pd{1, nullptr, d.gens, b->B, 1.0, 0.0};
        int64_t n_anti = 0, n_new = 0;
        float ms = 0;
        st = dress_pairs(ctx, pd, &n_anti, &n_new, &ms);
        if (st) return st;
        ctx->stats.n_dress++;
        ctx->stats.dressed_terms += M;
        ctx->stats.anticommuting += n_anti;
        ctx->stats.appended += n_new;
        ctx->stats.dress_kernel_ms += ms;
    }
    if (eps > 0) {
        CK(cudaMemsetAsync(ctx->counters.p, 0, kCountersClear, ctx->stream));
        int64_t removed = 0;
        st = compress(ctx, eps, 0, &removed);
        if (st) return st;
    }
    b->graph_M = -1;  // the Hamiltonians changed: capture again on the next screening
    if (energy_after || n_terms_after) {
        const int B = b->B;
        std::vector<double> e(B);
        std::vector<uint64_t> k(B), cnt(B);
        std::vector<double> g(B), abc(3 * (size_t)B), tau(B);
        std::vector<int64_t> nt(B);
        iqcc_batch_screen_out o2{e.data(), k.data(), cnt.data(), g.data(), abc.data(), tau.data(), nt.data()};
        st = batch_screen(b, theta, phi, &o2, false);
        if (st) return st;
        for (int p = 0; p < B; ++p) {
            if (energy_after) energy_after[p] = e[p];
            if (n_terms_after) n_terms_after[p] = nt[p];
        }
    }
    return IQCC_OK;
}

iqcc_status iqcc_batch_export(iqcc_batch* b, int problem, int64_t cap, int64_t* n, uint64_t* x, uint64_t* z,
                              double* coef) {
    if (!b) return fail(nullptr, IQCC_ERR_ARG, "null batch");
    iqcc_ctx* ctx = b->ctx;
    GUARD(ctx);
    if (!n || cap < 0 || problem < 0 || problem >= b->B) return fail(ctx, IQCC_ERR_ARG, "bad argument");
    const int64_t M = ctx->M;
    std::vector<uint64_t> ax((size_t)M), az((size_t)M);
    std::vector<double> ac((size_t)M);
    int64_t got = 0;
    iqcc_status st = iqcc_export(ctx, M, &got, ax.data(), az.data(), ac.data());
    if (st) return st;
    int64_t k = 0;
    for (int64_t i = 0; i < got; ++i) {
        if ((int)(az[i] >> kBatchTagShift) != problem) continue;
        if (k < cap) {
            if (!x || !z || !coef) return fail(ctx, IQCC_ERR_ARG, "null output array");
            x[k] = ax[i];
            z[k] = az[i] & kBatchXMask;
            coef[k] = ac[i];
        }
        ++k;
    }
    *n = k;
    return IQCC_OK;
}

iqcc_status iqcc_batch_get_info(const iqcc_batch* b, iqcc_batch_info* out) {
    if (!b || !out) return fail(nullptr, IQCC_ERR_ARG, "null argument");
    out->n_terms = b->ctx->M;
    out->screens = b->screens;
    out->graph_replays = b->replays;
    out->blocks_energy = b->blocks[0];
    out->blocks_group = b->blocks[1];
    out->blocks_abc = b->blocks[2];
    out->pad = 0;
    return IQCC_OK;
}

const char* iqcc_batch_last_error(const iqcc_batch* b) {
    if (!b) return g_last_error.c_str();
    return iqcc_last_error(b->ctx);
}

void iqcc_batch_free(iqcc_batch* b) {
    if (!b) return;
    if (b->gs) cudaStreamSynchronize(b->gs);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->ctx) {
        release(b->ctx, b->dev);
        release(b->ctx, b->groups);
        iqcc_free(b->ctx);
    }
    if (b->gs) cudaStreamDestroy(b->gs);
    if (b->h_occ) cudaFreeHost(b->h_occ);
    if (b->h_out) cudaFreeHost(b->h_out);
    cudaGetLastError();
    delete b;
}

}  // extern "C"

