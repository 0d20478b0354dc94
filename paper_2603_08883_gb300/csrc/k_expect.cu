// Expectation values over the QMF product state (Eq. 3 / Eq. 10):
//   energy   E = sum_T C_T <T>                                  (Eq. 12, tau = 0)
//   A, B, C  of E(tau) = A + B cos tau + C sin tau for one generator P
//            (Eq. 5 inserted into Eq. 12): A over commuting T, B over
//            anticommuting T, C = sum_anti C_T <i T P>
//   DIS      gradients g = dE/dtau at 0 (Eq. 7 / Eq. 13) of given candidate
//            generators at general angles (the candidates themselves and their
//            z-eigenstate gradients come from the flip-set grouping of
//            k_disgroup.cu).
//
// Two evaluation modes.
//  * Basis state (every theta_j in {0, pi}): <T> = 0 unless T has no X/Y, and
//    then <T> = (-1)^{popc(zT & occ)}.  No FP64 multiplies; only rows that can
//    contribute read their coefficient.
//  * General angles: per 4-qubit group a 256-entry table of products of the
//    single-qubit expectations <I>=1, <X>=sin th cos ph, <Y>=sin th sin ph,
//    <Z>=cos th, indexed by (x nibble << 4 | z nibble), kept in shared memory.
//
// Sums: per-thread FP64 accumulation, warp-shuffle and shared-memory block
// reduction, one partial per block, and a final fixed-order compensated sum -
// deterministic for a given launch shape.
#include <cuda_runtime.h>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;

template <int W>
__device__ __forceinline__ bool x_is_zero(const Key<W>& k) {
    uint64_t v = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) v |= k.x[j];
    return v == 0;
}

template <int W>
__device__ __forceinline__ bool x_equal(const Key<W>& a, const Key<W>& b) {
    uint64_t v = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) v |= a.x[j] ^ b.x[j];
    return v == 0;
}

// (-1)^{popc(z & occ)} for a string without X/Y.
template <int W>
__device__ __forceinline__ bool odd_occ(const Key<W>& k, const uint64_t* occ) {
    int s = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) s += __popcll(k.z[j] & occ[j]);
    return s & 1;
}

// Product of the per-group table entries: <Omega|P(k)|Omega>.
template <int W>
__device__ __forceinline__ double expect_tab(const Key<W>& k, const double* __restrict__ tab, int n_groups) {
    double v = 1.0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
#pragma unroll 4
        for (int q = 0; q < 16; ++q) {
            int g = j * 16 + q;
            if (g < n_groups) {
                unsigned xn = (unsigned)(k.x[j] >> (4 * q)) & 15u;
                unsigned zn = (unsigned)(k.z[j] >> (4 * q)) & 15u;
                v *= tab[g * 256 + (xn << 4 | zn)];
            }
        }
    }
    return v;
}

template <int N>
__device__ __forceinline__ void block_reduce_store(double (&v)[N], double* out) {
    __shared__ double red[kThreads / 32][N];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xFFFFFFFFu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) red[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x < N) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Dress-bin and per-tile counting folded into the A, B, C pass (see launch_abc).
struct PairCount {
    uint32_t* counts;
    uint32_t* tile_kept;
    int shift;
    int top_word;
    uint64_t top_mask;
    DevCounters* ctr;
};

// One row of the A, B, C pass: adds its share to acc; returns whether it
// anticommutes with p.
template <int W, bool BASIS>
__device__ __forceinline__ bool abc_row(const Key<W>& t, const double* __restrict__ coef, int64_t i, const Key<W>& p,
                                        int yP, const Key<W>& occ, const double* s_tab, int n_groups, double* acc) {
    const int anti = anticommutes<W>(t, p);
    if (BASIS) {
        const bool diag = x_is_zero<W>(t);
        const bool cross = anti && x_equal<W>(t, p);
        if (diag || cross) {
            const double c = coef[i];
            if (diag) {
                const double e = odd_occ<W>(t, occ.x) ? -c : c;
                if (anti) acc[1] += e;
                else acc[0] += e;
            }
            if (cross) {
                Key<W> q = key_xor<W>(t, p);
                const int s = product_sign<W>(t, yP, p, q);
                const bool neg = (s < 0) ^ odd_occ<W>(q, occ.x);
                acc[2] += neg ? -c : c;
            }
        }
    } else {
        const double c = coef[i];
        const double et = expect_tab<W>(t, s_tab, n_groups);
        if (anti) {
            acc[1] += c * et;
            Key<W> q = key_xor<W>(t, p);
            const int s = product_sign<W>(t, yP, p, q);
            acc[2] += (double)s * c * expect_tab<W>(q, s_tab, n_groups);
        } else {
            acc[0] += c * et;
        }
    }
    return anti != 0;
}

// A, B, C for generator p (p = 0: energy in A).  HIST: the same pass also
// counts, for the dress by p that follows (k_pairjoin.cu), the anticommuting
// rows and the commuting rows per tile of kDressTile rows (the blocks then
// walk whole tiles); one read of the keys for both.  The dress sizes its bins
// from the first count and places the commuting rows by the second.
template <int W, bool BASIS, bool HIST>
__global__ void __launch_bounds__(kThreads) k_abc(const uint64_t* __restrict__ rows,
                                                  const double* __restrict__ coef, int64_t M, Key<W> p,
                                                  int yP, Key<W> occ, const double* __restrict__ tables,
                                                  int n_groups, double* partials, PairCount pc,
                                                  const uint8_t* __restrict__ live) {
    extern __shared__ double s_tab[];
    if (!BASIS) {
        for (int i = threadIdx.x; i < n_groups * 256; i += blockDim.x) s_tab[i] = tables[i];
        __syncthreads();
    }
    double acc[3] = {0.0, 0.0, 0.0};
    if (HIST) {
        unsigned n_anti = 0;
        const int64_t n_tiles = (M + kDressTile - 1) / kDressTile;
        for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
            // the tile's rows of this thread in flight together: live flags, then keys
            constexpr int kPer = kDressTile / kThreads;
            bool v[kPer], k[kPer];
            Key<W> t[kPer];
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                const int64_t i = tile * kDressTile + r * kThreads + threadIdx.x;
                v[r] = i < M && (!live || live[i]);  // rows dropped by a pending term-limit cut are skipped
            }
#pragma unroll
            for (int r = 0; r < kPer; ++r)
                if (v[r]) t[r] = load_key<W>(rows, tile * kDressTile + r * kThreads + threadIdx.x);
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                const int64_t i = tile * kDressTile + r * kThreads + threadIdx.x;
                k[r] = false;
                if (!v[r]) continue;
                if (abc_row<W, BASIS>(t[r], coef, i, p, yP, occ, s_tab, n_groups, acc)) {
                    ++n_anti;
                } else {
                    k[r] = true;
                }
            }
            int kept = 0;
#pragma unroll
            for (int r = 0; r < kPer; ++r) kept += __syncthreads_count(k[r]);
            if (threadIdx.x == 0) pc.tile_kept[tile] = (uint32_t)kept;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n_anti += __shfl_down_sync(0xFFFFFFFFu, n_anti, o);
        if ((threadIdx.x & 31) == 0 && n_anti) atomicAdd(&pc.ctr->n_anti, (unsigned long long)n_anti);
    } else {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
            if (live && !live[i]) continue;  // dropped by a pending term-limit cut
            abc_row<W, BASIS>(load_key<W>(rows, i), coef, i, p, yP, occ, s_tab, n_groups, acc);
        }
    }
    block_reduce_store<3>(acc, partials + 3 * blockIdx.x);
}

// Fixed-order compensated sum of partials[n][3] -> out3.
__global__ void k_reduce3(const double* partials, int n, double* out3) {
    __shared__ double ss[kThreads][3];
    __shared__ double cc[kThreads][3];
    for (int k = 0; k < 3; ++k) {
        double s = 0.0, c = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double v = partials[3 * i + k];
            double t = s + v;
            c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
            s = t;
        }
        ss[threadIdx.x][k] = s;
        cc[threadIdx.x][k] = c;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        int k = threadIdx.x;
        double s = 0.0, c = 0.0;
        for (int i = 0; i < blockDim.x; ++i) {
            for (int part = 0; part < 2; ++part) {
                double v = part ? cc[i][k] : ss[i][k];
                double t = s + v;
                c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
                s = t;
            }
        }
        out3[k] = s + c;
    }
}

// Column sums of partials[rows][cols] (fixed order, compensated).
__global__ void k_reduce_cols(const double* partials, int rows, int cols, double* out) {
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= cols) return;
    double s = 0.0, c = 0.0;
    for (int r = 0; r < rows; ++r) {
        double v = partials[(size_t)r * cols + col];
        double t = s + v;
        c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    out[col] = s + c;
}

// tables[g][xn<<4|zn] = prod over the 4 qubits of the group of <sigma>.
__global__ void k_qmf_tables(const double* theta, const double* phi, int n, int n_groups, double* tables) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_groups * 256) return;
    int g = idx >> 8, e = idx & 255;
    unsigned xn = (unsigned)e >> 4, zn = (unsigned)e & 15u;
    double v = 1.0;
    for (int b = 0; b < 4; ++b) {
        int j = 4 * g + b;
        int xb = (xn >> b) & 1, zb = (zn >> b) & 1;
        if (!xb && !zb) continue;
        if (j >= n) { v = 0.0; continue; }          // no qubit there: such keys never occur
        double th = theta[j], ph = phi[j];
        bool basis = (th == 0.0) || (th == 3.141592653589793);
        double st = basis ? 0.0 : sin(th);
        double ct = cos(th);
        if (xb && !zb) v *= st * cos(ph);
        else if (xb && zb) v *= st * sin(ph);
        else v *= ct;
    }
    tables[idx] = v;
}

constexpr int kGradTile = 16;

// General-angle gradients of K (<= kGradTile) candidates:
// g_a = sum over T anticommuting with a of s C_T <P(T xor a)>.
template <int W>
__global__ void __launch_bounds__(kThreads) k_grad_general(const uint64_t* __restrict__ rows,
                                                           const double* __restrict__ coef, int64_t M,
                                                           const uint64_t* __restrict__ cand, int K,
                                                           const double* __restrict__ tables, int n_groups,
                                                           double* partials) {
    extern __shared__ double s_tab[];
    __shared__ Key<W> s_c[kGradTile];
    __shared__ int s_y[kGradTile];
    for (int i = threadIdx.x; i < n_groups * 256; i += blockDim.x) s_tab[i] = tables[i];
    if (threadIdx.x < K) {
        Key<W> a;
        int y = 0;
        for (int j = 0; j < W; ++j) {
            a.x[j] = cand[threadIdx.x * 2 * W + j];
            a.z[j] = cand[threadIdx.x * 2 * W + W + j];
            y += __popcll(a.x[j] & a.z[j]);
        }
        s_c[threadIdx.x] = a;
        s_y[threadIdx.x] = y & 3;
    }
    __syncthreads();
    double acc[kGradTile];
#pragma unroll
    for (int k = 0; k < kGradTile; ++k) acc[k] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        Key<W> t = load_key<W>(rows, i);
        const double c = coef[i];
#pragma unroll
        for (int k = 0; k < kGradTile; ++k) {
            if (k < K && anticommutes<W>(t, s_c[k])) {
                Key<W> q = key_xor<W>(t, s_c[k]);
                const int s = product_sign<W>(t, s_y[k], s_c[k], q);
                acc[k] += (double)s * c * expect_tab<W>(q, s_tab, n_groups);
            }
        }
    }
    block_reduce_store<kGradTile>(acc, partials + (size_t)kGradTile * blockIdx.x);
}

template <int W>
Key<W> key_from(const uint64_t* w) {
    Key<W> k;
    for (int j = 0; j < W; ++j) { k.x[j] = w[j]; k.z[j] = w[W + j]; }
    return k;
}

int abc_grid(int64_t M) {
    int64_t want = (M + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)sm_count() * 4;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

template <int W, bool HIST>
void abc_launch(const uint64_t* rows, const double* coef, int64_t M, const Key<W>& p, int y, const Key<W>& occ,
                bool basis, const double* tables, int n_groups, double* partials, const PairCount& pc,
                const uint8_t* live, cudaStream_t s) {
    const int grid = expect_blocks();
    if (basis) {
        k_abc<W, true, HIST><<<grid, kThreads, 0, s>>>(rows, coef, M, p, y & 3, occ, tables, n_groups, partials, pc,
                                                        live);
    } else {
        size_t smem = (size_t)n_groups * 256 * sizeof(double);
        static std::atomic<unsigned long long> attr{0};
        if (first_on_device(&attr))
            cudaFuncSetAttribute(k_abc<W, false, HIST>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 256 * 8);
        k_abc<W, false, HIST><<<grid, kThreads, smem, s>>>(rows, coef, M, p, y & 3, occ, tables, n_groups, partials,
                                                            pc, live);
    }
    note_launch();
}

template <int W>
void abc_impl(const uint64_t* rows, const double* coef, int64_t M, const uint64_t* pkey, bool basis,
              const uint64_t* occ_words, const double* tables, int n_groups, double* partials, cudaStream_t s,
              const PairHistOut* pair, const uint8_t* live) {
    Key<W> p = key_from<W>(pkey);
    int y = 0;
    for (int j = 0; j < W; ++j) y += __builtin_popcountll(p.x[j] & p.z[j]);
    Key<W> occ{};
    for (int j = 0; j < W; ++j) { occ.x[j] = occ_words[j]; occ.z[j] = 0; }
    PairCount pc{};
    if (pair) {
        const Gen<W> g = make_gen<W>(pkey, 1.0, 0.0);
        pc = PairCount{pair->counts, pair->tile_kept, 64 - pair->log2_bins, g.top_word, g.top_mask, pair->ctr};
        abc_launch<W, true>(rows, coef, M, p, y, occ, basis, tables, n_groups, partials, pc, live, s);
    } else {
        abc_launch<W, false>(rows, coef, M, p, y, occ, basis, tables, n_groups, partials, pc, live, s);
    }
}

template <int W>
void grad_impl(const uint64_t* rows, const double* coef, int64_t M, const uint64_t* cand, int K,
               const double* tables, int n_groups, double* partials, int n_blocks, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    if (first_on_device(&attr))
        cudaFuncSetAttribute(k_grad_general<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 256 * 8);
    size_t smem = (size_t)n_groups * 256 * sizeof(double);
    k_grad_general<W><<<n_blocks, kThreads, smem, s>>>(rows, coef, M, cand, K, tables, n_groups, partials); note_launch();
}

}  // namespace

int expect_blocks() { return sm_count() * 4; }

void launch_abc(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* pkey, bool basis,
                const uint64_t* occ, const double* tables, int n_groups, double* partials, cudaStream_t s,
                const PairHistOut* pair, const uint8_t* live) {
    switch (Wd) {
        case 1: abc_impl<1>(rows, coef, M, pkey, basis, occ, tables, n_groups, partials, s, pair, live); break;
        case 2: abc_impl<2>(rows, coef, M, pkey, basis, occ, tables, n_groups, partials, s, pair, live); break;
        default: abc_impl<4>(rows, coef, M, pkey, basis, occ, tables, n_groups, partials, s, pair, live); break;
    }
}

void launch_reduce3(const double* partials, int n, double* out3, cudaStream_t s) {
    k_reduce3<<<1, kThreads, 0, s>>>(partials, n, out3); note_launch();
}

void launch_reduce_cols(const double* partials, int rows, int cols, double* out, cudaStream_t s) {
    k_reduce_cols<<<(cols + 127) / 128, 128, 0, s>>>(partials, rows, cols, out); note_launch();
}

void launch_qmf_tables(const double* theta, const double* phi, int n, int n_groups, double* tables,
                       cudaStream_t s) {
    int total = n_groups * 256;
    k_qmf_tables<<<(total + 255) / 256, 256, 0, s>>>(theta, phi, n, n_groups, tables); note_launch();
}

void launch_grad_general(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* cand,
                         int K, const double* tables, int n_groups, double* partials, int n_blocks,
                         cudaStream_t s) {
    switch (Wd) {
        case 1: grad_impl<1>(rows, coef, M, cand, K, tables, n_groups, partials, n_blocks, s); break;
        case 2: grad_impl<2>(rows, coef, M, cand, K, tables, n_groups, partials, n_blocks, s); break;
        default: grad_impl<4>(rows, coef, M, cand, K, tables, n_groups, partials, n_blocks, s); break;
    }
}

}  // namespace iqcc
