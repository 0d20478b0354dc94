// Sort-based dressing: the alternative to the hash merge of k_dress.cu.
//
// A group of k generators (Eq. 6, applied in order) is expanded without
// merging: every row T follows every path through the group, where at
// generator j a path either keeps the current string S (factor cos tau_j if S
// anticommutes with P_j, else 1) or, only when S anticommutes with P_j, moves
// to the partner S xor P_j with factor s sin tau_j (iSP_j = s (S xor P_j),
// Eq. 5 in the library sign).  Summing the leaves by key gives the group's
// dressed Hamiltonian (the merge of App. D, Eq. 18, done once per group by a
// radix sort and a segmented sum instead of a lookup per generator).  Paths
// are enumerated as k-bit masks (bit j set: partner branch at generator j).
#include <cuda_runtime.h>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxFuse = 8;

template <int W>
struct GenGroup {
    Key<W> p[kMaxFuse];
    int yP[kMaxFuse];
    double cos_t[kMaxFuse], sin_t[kMaxFuse];
    int k;
};

// Follows path `mask` from t; false when the path takes a partner branch at a
// generator its current string commutes with.
template <int W>
__device__ __forceinline__ bool follow(const GenGroup<W>& g, Key<W> t, unsigned mask, Key<W>* leaf, double* factor) {
    double f = 1.0;
    for (int j = 0; j < g.k; ++j) {
        const bool anti = anticommutes<W>(t, g.p[j]) != 0;
        const bool jump = (mask >> j) & 1u;
        if (jump && !anti) return false;
        if (!anti) continue;
        if (jump) {
            const Key<W> q = key_xor<W>(t, g.p[j]);
            f *= (double)product_sign<W>(t, g.yP[j], g.p[j], q) * g.sin_t[j];
            t = q;
        } else {
            f *= g.cos_t[j];
        }
    }
    *leaf = t;
    *factor = f;
    return true;
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_expand_count(const uint64_t* __restrict__ rows, int64_t M,
                                                           GenGroup<W> g, unsigned long long* total) {
    unsigned long long cnt = 0;
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += s) {
        const Key<W> t = load_key<W>(rows, i);
        for (unsigned mask = 0; mask < (1u << g.k); ++mask) {
            Key<W> leaf;
            double f;
            cnt += follow<W>(g, t, mask, &leaf, &f) ? 1 : 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(total, cnt);
}

// Leaves of every row appended at out[*next ...] (warp-aggregated), at most cap.
template <int W>
__global__ void __launch_bounds__(kThreads) k_expand_emit(const uint64_t* __restrict__ rows,
                                                          const double* __restrict__ coef, int64_t M, GenGroup<W> g,
                                                          uint64_t* out_rows, double* out_coef,
                                                          unsigned long long* next, int64_t cap, DevCounters* ctr) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // every lane of a warp runs the same number of iterations (ballots below)
    for (int64_t base = i0 - lane; base < M; base += s) {
        const int64_t i = base + lane;
        const bool live = i < M;
        Key<W> t{};
        double c = 0.0;
        if (live) {
            t = load_key<W>(rows, i);
            c = coef[i];
        }
        for (unsigned mask = 0; mask < (1u << g.k); ++mask) {
            Key<W> leaf{};
            double f = 0.0;
            const bool ok = live && follow<W>(g, t, mask, &leaf, &f);
            const unsigned b = __ballot_sync(FULL, ok);
            if (!b) continue;
            const int leader = __ffs(b) - 1;
            unsigned long long at = 0;
            if (lane == leader) at = atomicAdd(next, (unsigned long long)__popc(b));
            at = __shfl_sync(FULL, at, leader) + __popc(b & lt);
            if (ok) {
                if ((int64_t)at < cap) {
                    store_key<W>(out_rows, (int64_t)at, leaf);
                    out_coef[at] = c * f;
                } else {
                    set_error(ctr, IQCC_ERR_STATE, 30);
                }
            }
        }
    }
}

// E_fut(T) = <Omega| D_k ... D_1 (T) |Omega>: the energy of the single string T
// after the group's generators (Eq. 5, Eq. 12), summed over T's paths (each
// leaf's factor times its expectation, a product of per-qubit <sigma> from
// tab[ts k + letter], letter 1..3 = X, Y, Z).  By linearity of the dress, deleting T from H now changes
// the energy after those generators by exactly -C_T E_fut(T).
template <int W>
__global__ void __launch_bounds__(kThreads) k_future_energy(const uint64_t* __restrict__ rows, int64_t M, GenGroup<W> g,
                                                            const double* __restrict__ tab_g, int ts, int n,
                                                            double* out) {
    extern __shared__ double tab[];
    for (int i = threadIdx.x; i < ts * n; i += blockDim.x) tab[i] = tab_g[i];
    __syncthreads();
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += s) {
        const Key<W> t = load_key<W>(rows, i);
        double e = 0.0;
        for (unsigned mask = 0; mask < (1u << g.k); ++mask) {
            Key<W> leaf;
            double f;
            if (!follow<W>(g, t, mask, &leaf, &f)) continue;
            double v = f;
#pragma unroll
            for (int wd = 0; wd < W && v != 0.0; ++wd) {
                uint64_t m = leaf.x[wd] | leaf.z[wd];
                while (m && v != 0.0) {
                    const int j = __ffsll((long long)m) - 1;
                    m &= m - 1;
                    const int xb = (int)((leaf.x[wd] >> j) & 1ull), zb = (int)((leaf.z[wd] >> j) & 1ull);
                    v *= tab[ts * (64 * wd + j) + (xb ? (zb ? 2 : 1) : 3)];
                }
            }
            e += v;
        }
        out[i] = e;
    }
}

template <int W>
GenGroup<W> make_group(const uint64_t* pkeys, const double* tau, int k) {
    GenGroup<W> g{};
    g.k = k;
    for (int j = 0; j < k; ++j) {
        int y = 0;
        for (int w = 0; w < W; ++w) {
            g.p[j].x[w] = pkeys[(size_t)j * 2 * W + w];
            g.p[j].z[w] = pkeys[(size_t)j * 2 * W + W + w];
            y += __builtin_popcountll(g.p[j].x[w] & g.p[j].z[w]);
        }
        g.yP[j] = y & 3;
        g.cos_t[j] = std::cos(tau[j]);
        g.sin_t[j] = std::sin(tau[j]);
    }
    return g;
}

int expand_grid(int64_t M) {
    int64_t want = (M + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

}  // namespace

int max_fuse() { return kMaxFuse; }

void launch_future_energy(int Wd, const uint64_t* rows, int64_t M, const uint64_t* pkeys, const double* tau, int k,
                          const double* tab, int ts, int n, double* out, cudaStream_t s) {
    if (M <= 0) return;
    const int g = expand_grid(M);
    const size_t smem = (size_t)ts * n * sizeof(double);
    switch (Wd) {
        case 1: k_future_energy<1><<<g, kThreads, smem, s>>>(rows, M, make_group<1>(pkeys, tau, k), tab, ts, n, out); break;
        case 2: k_future_energy<2><<<g, kThreads, smem, s>>>(rows, M, make_group<2>(pkeys, tau, k), tab, ts, n, out); break;
        default: k_future_energy<4><<<g, kThreads, smem, s>>>(rows, M, make_group<4>(pkeys, tau, k), tab, ts, n, out); break;
    }
    note_launch();
}

void launch_expand_count(int Wd, const uint64_t* rows, int64_t M, const uint64_t* pkeys, const double* tau, int k,
                         unsigned long long* total, cudaStream_t s) {
    if (M <= 0) return;
    const int g = expand_grid(M);
    switch (Wd) {
        case 1: k_expand_count<1><<<g, kThreads, 0, s>>>(rows, M, make_group<1>(pkeys, tau, k), total); break;
        case 2: k_expand_count<2><<<g, kThreads, 0, s>>>(rows, M, make_group<2>(pkeys, tau, k), total); break;
        default: k_expand_count<4><<<g, kThreads, 0, s>>>(rows, M, make_group<4>(pkeys, tau, k), total); break;
    }
    note_launch();
}

void launch_expand_emit(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* pkeys,
                        const double* tau, int k, uint64_t* out_rows, double* out_coef, unsigned long long* next,
                        int64_t cap, DevCounters* ctr, cudaStream_t s) {
    if (M <= 0) return;
    const int g = expand_grid(M);
    switch (Wd) {
        case 1:
            k_expand_emit<1><<<g, kThreads, 0, s>>>(rows, coef, M, make_group<1>(pkeys, tau, k), out_rows, out_coef,
                                                     next, cap, ctr);
            break;
        case 2:
            k_expand_emit<2><<<g, kThreads, 0, s>>>(rows, coef, M, make_group<2>(pkeys, tau, k), out_rows, out_coef,
                                                     next, cap, ctr);
            break;
        default:
            k_expand_emit<4><<<g, kThreads, 0, s>>>(rows, coef, M, make_group<4>(pkeys, tau, k), out_rows, out_coef,
                                                     next, cap, ctr);
            break;
    }
    note_launch();
}

}  // namespace iqcc
