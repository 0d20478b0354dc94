// Adjoint of the QMF energy: derivatives of the dressed energy with respect to
// the product-state angles (Eq. 3) and to the amplitude of one generator.
//
// For a generator P at amplitude tau (library sign, dress = e^{-i tau P/2} H
// e^{+i tau P/2}), Eq. 5 inserted into Eq. 12 gives E(tau) = A + B cos tau +
// C sin tau, with A the commuting terms' sum of C_T <T>, B the anticommuting
// terms' sum of C_T <T> and C their sum of s_T C_T <Q>, Q = T xor P and
// iTP = s_T Q.  Every <S> is a product over the qubits of S of single-qubit
// expectations (<X> = sin t cos p, <Y> = sin t sin p, <Z> = cos t), so
//   dE/dt_k = sum over commuting T of C_T d<T>/dt_k
//           + cos tau * sum over anticommuting T of C_T d<T>/dt_k
//           + sin tau * sum over anticommuting T of s_T C_T d<Q>/dt_k,
// and likewise for p_k; d<S>/dt_k is qubit k's derivative times the product
// of the other qubits' factors.  dE/dtau = -B sin tau + C cos tau.  Without a
// generator every term commutes and the pass gives E and its angle gradient.
//
// For a z-eigenstate (every theta 0 or pi) X and Y factors vanish and Z
// factors are +-1, so a string with two or more flipped qubits contributes
// nothing, a diagonal one only its sign (and no angle derivative), and one
// with a single flipped qubit k only d/dtheta_k: popcounts and signs, at most
// one atomic add per string.  For general angles the derivative of <S> at
// qubit k is <S> times the ratio d<sigma_k>/<sigma_k> (tabulated per qubit and
// letter) when no factor of S is zero, so each string adds w C <S> to one sum
// S_k(sigma) per support qubit, and dE/dt_k = sum over sigma of the theta ratio
// times S_k(sigma) (likewise for p) in a final combination; a string with
// exactly one zero factor (at k0) adds w C times the product of its other
// factors times the derivative at k0 directly; two or more zero factors: none.
// Block sums live in shared memory (FP64 atomic adds) and are reduced column by
// column.
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>
#include <cuda_runtime.h>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;

// Per-qubit table, kTab doubles: [0..3] <sigma> (I, X, Y, Z), [4..7] d/dt,
// [8..11] d/dp, [12..14] d/dt over <sigma> (X, Y, Z; 0 where <sigma> = 0),
// [15..17] d/dp over <sigma>.  A z-eigenstate qubit (t = 0 or pi) takes
// sin t = 0 exactly.
constexpr int kTab = 18;

__global__ void k_grad_tables(const double* theta, const double* phi, int n, double* tab) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double t = theta[k], p = phi[k];
    const bool basis = (t == 0.0) || (t == 3.141592653589793);
    const double st = basis ? 0.0 : sin(t), ct = cos(t), sp = sin(p), cp = cos(p);
    double* r = tab + kTab * k;
    r[0] = 1.0;      r[1] = st * cp;   r[2] = st * sp;  r[3] = ct;
    r[4] = 0.0;      r[5] = ct * cp;   r[6] = ct * sp;  r[7] = -st;
    r[8] = 0.0;      r[9] = -st * sp;  r[10] = st * cp; r[11] = 0.0;
    for (int l = 1; l <= 3; ++l) {
        r[11 + l] = r[l] != 0.0 ? r[4 + l] / r[l] : 0.0;
        r[14 + l] = r[l] != 0.0 ? r[8 + l] / r[l] : 0.0;
    }
}

// Column layout of the block partials: S_k(sigma) at 3k + sigma - 1, the direct
// d/dt sums at 3n + k, the direct d/dp sums at 4n + k, then A, B, C.
__host__ __device__ __forceinline__ int grad_cols(int n) { return 5 * n + 3; }

struct LetterMasks {
    uint64_t zero[3][4];    // qubits whose <X>, <Y>, <Z> is exactly zero
    uint64_t useful[3][4];  // qubits whose X, Y, Z ratio (theta or phi) is non-zero
};

template <int W>
__device__ __forceinline__ void letters(const Key<W>& s, int wd, uint64_t* xo, uint64_t* yy, uint64_t* zo) {
    *xo = s.x[wd] & ~s.z[wd];
    *yy = s.x[wd] & s.z[wd];
    *zo = s.z[wd] & ~s.x[wd];
}

// Product of the non-zero factors of letter l (1..3) on the qubits of mask b in
// word wd; a qubit whose factor is zero is reported in *k0, *l0 instead.
__device__ __forceinline__ double letter_product(uint64_t b, int wd, int l, uint64_t zero, const double* tab, int* k0,
                                                 int* l0) {
    const uint64_t zb = b & zero;
    if (zb) {
        *k0 = 64 * wd + __ffsll((long long)zb) - 1;
        *l0 = l;
        b &= ~zb;
    }
    double prod = 1.0;
    while (b) {
        const int k = 64 * wd + __ffsll((long long)b) - 1;
        b &= b - 1;
        prod *= tab[kTab * k + l];
    }
    return prod;
}

// v added to S_k(letter li) (li = 0..2) for the qubits of mask b in word wd.
__device__ __forceinline__ void letter_sums(uint64_t b, int wd, int li, double v, double* acc) {
    while (b) {
        const int k = 64 * wd + __ffsll((long long)b) - 1;
        b &= b - 1;
        atomicAdd(acc + 3 * k + li, v);
    }
}

// General angles: <S> (0 when a factor vanishes) and the string's
// contributions w C d<S> to the block sums (w C given as wc).
template <int W>
__device__ __forceinline__ double string_general(const Key<W>& s, double wc, const double* tab, const LetterMasks& m,
                                                 double* acc, int n) {
    int zeros = 0;
#pragma unroll
    for (int wd = 0; wd < W; ++wd) {
        uint64_t xo, yy, zo;
        letters<W>(s, wd, &xo, &yy, &zo);
        zeros += __popcll(xo & m.zero[0][wd]) + __popcll(yy & m.zero[1][wd]) + __popcll(zo & m.zero[2][wd]);
    }
    if (zeros >= 2) return 0.0;
    double prod = 1.0;
    int k0 = -1, l0 = 0;
#pragma unroll
    for (int wd = 0; wd < W; ++wd) {
        uint64_t xo, yy, zo;
        letters<W>(s, wd, &xo, &yy, &zo);
        prod *= letter_product(xo, wd, 1, m.zero[0][wd], tab, &k0, &l0);
        prod *= letter_product(yy, wd, 2, m.zero[1][wd], tab, &k0, &l0);
        prod *= letter_product(zo, wd, 3, m.zero[2][wd], tab, &k0, &l0);
    }
    if (wc == 0.0) return zeros ? 0.0 : prod;
    if (zeros == 1) {
        const double dt = tab[kTab * k0 + 4 + l0], dp = tab[kTab * k0 + 8 + l0];
        if (dt != 0.0) atomicAdd(acc + 3 * n + k0, wc * prod * dt);
        if (dp != 0.0) atomicAdd(acc + 4 * n + k0, wc * prod * dp);
        return 0.0;
    }
    const double v = wc * prod;
#pragma unroll
    for (int wd = 0; wd < W; ++wd) {
        uint64_t xo, yy, zo;
        letters<W>(s, wd, &xo, &yy, &zo);
        letter_sums(xo & m.useful[0][wd], wd, 0, v, acc);
        letter_sums(yy & m.useful[1][wd], wd, 1, v, acc);
        letter_sums(zo & m.useful[2][wd], wd, 2, v, acc);
    }
    return prod;
}

// z-eigenstate: <S> and the single-flip contribution, from popcounts.
template <int W>
__device__ __forceinline__ double string_basis(const Key<W>& s, double wc, const double* tab, const Key<W>& occ,
                                               double* acc, int n) {
    int flips = 0, neg = 0, k0 = -1, l0 = 1;
#pragma unroll
    for (int wd = 0; wd < W; ++wd) {
        flips += __popcll(s.x[wd]);
        if (s.x[wd]) {
            const int j = __ffsll((long long)s.x[wd]) - 1;
            k0 = 64 * wd + j;
            l0 = ((s.z[wd] >> j) & 1ull) ? 2 : 1;  // Y or X
        }
    }
    if (flips >= 2) return 0.0;
#pragma unroll
    for (int wd = 0; wd < W; ++wd) neg += __popcll(s.z[wd] & ~s.x[wd] & occ.x[wd]);
    const double sign = (neg & 1) ? -1.0 : 1.0;
    if (flips == 0) return sign;
    if (wc != 0.0) {
        const double dt = tab[kTab * k0 + 4 + l0];
        if (dt != 0.0) {
            // single-flip strings pile onto few qubits: lanes with the same
            // qubit sum their terms first, one shared-memory atomic per qubit
            namespace cg = cooperative_groups;
            const cg::coalesced_group g = cg::coalesced_threads();
            const cg::coalesced_group same = cg::labeled_partition(g, k0);
            const double sum = cg::reduce(same, wc * sign * dt, cg::plus<double>());
            if (same.thread_rank() == 0) atomicAdd(acc + 3 * n + k0, sum);
        }
    }
    return 0.0;
}

template <int W, bool BASIS>
__global__ void __launch_bounds__(kThreads) k_energy_grad(const uint64_t* __restrict__ rows,
                                                          const double* __restrict__ coef, int64_t M, Key<W> p, int yP,
                                                          bool has_gen, double cos_t, double sin_t,
                                                          const double* __restrict__ tab_g, int n, Key<W> occ,
                                                          double* partials) {
    extern __shared__ double sm[];
    double* tab = sm;              // kTab n
    double* acc = sm + kTab * n;   // grad_cols(n)
    __shared__ LetterMasks s_m;
    const int cols = grad_cols(n);
    for (int i = threadIdx.x; i < kTab * n; i += blockDim.x) tab[i] = tab_g[i];
    for (int i = threadIdx.x; i < cols; i += blockDim.x) acc[i] = 0.0;
    if (threadIdx.x < 24) (&s_m.zero[0][0])[threadIdx.x] = 0ull;
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double* r = tab_g + kTab * k;
        for (int l = 0; l < 3; ++l) {
            const unsigned long long bit = 1ull << (k % 64);
            if (r[l + 1] == 0.0) atomicOr((unsigned long long*)&s_m.zero[l][k / 64], bit);
            if (r[12 + l] != 0.0 || r[15 + l] != 0.0) atomicOr((unsigned long long*)&s_m.useful[l][k / 64], bit);
        }
    }
    __syncthreads();
    const LetterMasks& m = s_m;
    double a = 0.0, b = 0.0, c = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        const Key<W> t = load_key<W>(rows, i);
        const double ct = coef[i];
        if (!has_gen || !anticommutes<W>(t, p)) {
            a += ct * (BASIS ? string_basis<W>(t, ct, tab, occ, acc, n) : string_general<W>(t, ct, tab, m, acc, n));
        } else {
            b += ct * (BASIS ? string_basis<W>(t, cos_t * ct, tab, occ, acc, n)
                             : string_general<W>(t, cos_t * ct, tab, m, acc, n));
            const Key<W> q = key_xor<W>(t, p);
            const double s = (double)product_sign<W>(t, yP, p, q);
            c += s * ct * (BASIS ? string_basis<W>(q, sin_t * s * ct, tab, occ, acc, n)
                                 : string_general<W>(q, sin_t * s * ct, tab, m, acc, n));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xFFFFFFFFu, a, o);
        b += __shfl_down_sync(0xFFFFFFFFu, b, o);
        c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc + 5 * n, a);
        atomicAdd(acc + 5 * n + 1, b);
        atomicAdd(acc + 5 * n + 2, c);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cols; i += blockDim.x) partials[(size_t)blockIdx.x * cols + i] = acc[i];
}

// dE/dt_k = sum_sigma ratio_t(k, sigma) S_k(sigma) + direct; likewise for p.
// out: [0, n) d/dt, [n, 2n) d/dp, [2n, 2n + 3) A, B, C.
__global__ void k_grad_combine(const double* sums, const double* tab, int n, double* out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 3) out[2 * n + k] = sums[5 * n + k];
    if (k >= n) return;
    double gt = sums[3 * n + k], gp = sums[4 * n + k];
    for (int l = 0; l < 3; ++l) {
        const double sk = sums[3 * k + l];
        if (sk == 0.0) continue;
        gt += tab[kTab * k + 12 + l] * sk;
        gp += tab[kTab * k + 15 + l] * sk;
    }
    out[k] = gt;
    out[n + k] = gp;
}

template <int W>
void launch_w(const uint64_t* rows, const double* coef, int64_t M, const uint64_t* pkey, bool has_gen, double cos_t,
              double sin_t, const double* tab, int n, const uint64_t* occ_words, bool basis, double* partials,
              int blocks, cudaStream_t s) {
    Key<W> p{}, occ{};
    int y = 0;
    for (int j = 0; j < W; ++j) {
        p.x[j] = has_gen ? pkey[j] : 0ull;
        p.z[j] = has_gen ? pkey[W + j] : 0ull;
        y += __builtin_popcountll(p.x[j] & p.z[j]);
        occ.x[j] = occ_words[j];
    }
    const size_t smem = (size_t)(kTab * n + grad_cols(n)) * sizeof(double);
    if (basis)
        k_energy_grad<W, true><<<blocks, kThreads, smem, s>>>(rows, coef, M, p, y & 3, has_gen, cos_t, sin_t, tab, n,
                                                               occ, partials);
    else
        k_energy_grad<W, false><<<blocks, kThreads, smem, s>>>(rows, coef, M, p, y & 3, has_gen, cos_t, sin_t, tab,
                                                                n, occ, partials);
}

}  // namespace

int energy_grad_blocks() { return sm_count() * 4; }
int energy_grad_table_doubles(int n) { return kTab * n; }
int energy_grad_cols(int n) { return grad_cols(n); }

void launch_grad_tables(const double* theta, const double* phi, int n, double* tab, cudaStream_t s) {
    k_grad_tables<<<(n + 127) / 128, 128, 0, s>>>(theta, phi, n, tab);
    note_launch();
}

void launch_energy_grad(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* pkey,
                        bool has_gen, double cos_t, double sin_t, const double* tab, int n, const uint64_t* occ_words,
                        bool basis, double* partials, int blocks, cudaStream_t s) {
    switch (Wd) {
        case 1: launch_w<1>(rows, coef, M, pkey, has_gen, cos_t, sin_t, tab, n, occ_words, basis, partials, blocks, s); break;
        case 2: launch_w<2>(rows, coef, M, pkey, has_gen, cos_t, sin_t, tab, n, occ_words, basis, partials, blocks, s); break;
        default: launch_w<4>(rows, coef, M, pkey, has_gen, cos_t, sin_t, tab, n, occ_words, basis, partials, blocks, s); break;
    }
    note_launch();
}

void launch_grad_combine(const double* sums, const double* tab, int n, double* out, cudaStream_t s) {
    k_grad_combine<<<(n + 127) / 128, 128, 0, s>>>(sums, tab, n, out);
    note_launch();
}

}  // namespace iqcc
