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
// of the other qubits' factors.  That product is taken as the product of the
// non-zero factors of S divided by qubit k's (exact zeros counted apart: with
// two or more zero factors every derivative of S vanishes, with one only the
// zero qubit's survives).  dE/dtau = -B sin tau + C cos tau.  Without a
// generator every term commutes and the pass gives E and its angle gradient.
//
// One streaming pass over the rows; per block, the 2n gradient sums live in
// shared memory (FP64 atomic adds, skipped where the derivative is zero: at a
// z-eigenstate only strings with at most one flipped qubit reach them) and
// A, B, C in registers; block partials are reduced column by column.
#include <cuda_runtime.h>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;

// Per-qubit table: [k][0..3] <sigma>, [k][4..7] d<sigma>/dt, [k][8..11] d<sigma>/dp,
// sigma = I, X, Y, Z.  A z-eigenstate qubit (t = 0 or pi) takes sin t = 0 exactly.
__global__ void k_grad_tables(const double* theta, const double* phi, int n, double* tab) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double t = theta[k], p = phi[k];
    const bool basis = (t == 0.0) || (t == 3.141592653589793);
    const double st = basis ? 0.0 : sin(t), ct = cos(t), sp = sin(p), cp = cos(p);
    double* r = tab + 12 * k;
    r[0] = 1.0;      r[1] = st * cp;   r[2] = st * sp;  r[3] = ct;
    r[4] = 0.0;      r[5] = ct * cp;   r[6] = ct * sp;  r[7] = -st;
    r[8] = 0.0;      r[9] = -st * sp;  r[10] = st * cp; r[11] = 0.0;
}

__device__ __forceinline__ int letter_of(uint64_t x, uint64_t z, int j) {
    const int xb = (int)((x >> j) & 1ull), zb = (int)((z >> j) & 1ull);
    return xb ? (zb ? 2 : 1) : 3;  // X, Y or Z (called on support bits only)
}

// <S> of string S (x, z words) and, when w != 0, w * d<S>/dt_k and w * d<S>/dp_k
// added to acc[k] and acc[n + k].
template <int W>
__device__ __forceinline__ double string_adjoint(const Key<W>& s, double w, const double* tab, double* acc, int n) {
    double prod = 1.0;
    int zeros = 0, zk = -1, zl = 0;
#pragma unroll
    for (int wd = 0; wd < W; ++wd) {
        uint64_t m = s.x[wd] | s.z[wd];
        while (m) {
            const int j = __ffsll((long long)m) - 1;
            m &= m - 1;
            const int k = 64 * wd + j;
            const int l = letter_of(s.x[wd], s.z[wd], j);
            const double v = tab[12 * k + l];
            if (v == 0.0) {
                ++zeros;
                zk = k;
                zl = l;
            } else {
                prod *= v;
            }
        }
    }
    if (w == 0.0 || zeros >= 2) return zeros ? 0.0 : prod;
    if (zeros == 1) {
        const double dt = tab[12 * zk + 4 + zl], dp = tab[12 * zk + 8 + zl];
        if (dt != 0.0) atomicAdd(acc + zk, w * prod * dt);
        if (dp != 0.0) atomicAdd(acc + n + zk, w * prod * dp);
        return 0.0;
    }
#pragma unroll
    for (int wd = 0; wd < W; ++wd) {
        uint64_t m = s.x[wd] | s.z[wd];
        while (m) {
            const int j = __ffsll((long long)m) - 1;
            m &= m - 1;
            const int k = 64 * wd + j;
            const int l = letter_of(s.x[wd], s.z[wd], j);
            const double dt = tab[12 * k + 4 + l], dp = tab[12 * k + 8 + l];
            if (dt == 0.0 && dp == 0.0) continue;
            const double others = prod / tab[12 * k + l];
            if (dt != 0.0) atomicAdd(acc + k, w * others * dt);
            if (dp != 0.0) atomicAdd(acc + n + k, w * others * dp);
        }
    }
    return prod;
}

// partials[block][0..n) dE/dt, [n..2n) dE/dp, [2n..2n+3) A, B, C.
template <int W>
__global__ void __launch_bounds__(kThreads) k_energy_grad(const uint64_t* __restrict__ rows,
                                                          const double* __restrict__ coef, int64_t M, Key<W> p, int yP,
                                                          bool has_gen, double cos_t, double sin_t,
                                                          const double* __restrict__ tab_g, int n, double* partials) {
    extern __shared__ double sm[];
    double* tab = sm;           // 12 n
    double* acc = sm + 12 * n;  // 2 n + 3
    const int cols = 2 * n + 3;
    for (int i = threadIdx.x; i < 12 * n; i += blockDim.x) tab[i] = tab_g[i];
    for (int i = threadIdx.x; i < cols; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    double a = 0.0, b = 0.0, c = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        const Key<W> t = load_key<W>(rows, i);
        const double ct = coef[i];
        if (!has_gen || !anticommutes<W>(t, p)) {
            a += ct * string_adjoint<W>(t, ct, tab, acc, n);
        } else {
            b += ct * string_adjoint<W>(t, cos_t * ct, tab, acc, n);
            const Key<W> q = key_xor<W>(t, p);
            const double s = (double)product_sign<W>(t, yP, p, q);
            c += s * ct * string_adjoint<W>(q, sin_t * s * ct, tab, acc, n);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xFFFFFFFFu, a, o);
        b += __shfl_down_sync(0xFFFFFFFFu, b, o);
        c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc + 2 * n, a);
        atomicAdd(acc + 2 * n + 1, b);
        atomicAdd(acc + 2 * n + 2, c);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cols; i += blockDim.x) partials[(size_t)blockIdx.x * cols + i] = acc[i];
}

template <int W>
void launch_w(const uint64_t* rows, const double* coef, int64_t M, const uint64_t* pkey, bool has_gen, double cos_t,
              double sin_t, const double* tab, int n, double* partials, int blocks, cudaStream_t s) {
    Key<W> p{};
    int y = 0;
    for (int j = 0; j < W; ++j) {
        p.x[j] = has_gen ? pkey[j] : 0ull;
        p.z[j] = has_gen ? pkey[W + j] : 0ull;
        y += __builtin_popcountll(p.x[j] & p.z[j]);
    }
    const size_t smem = (size_t)(12 * n + 2 * n + 3) * sizeof(double);
    k_energy_grad<W><<<blocks, kThreads, smem, s>>>(rows, coef, M, p, y & 3, has_gen, cos_t, sin_t, tab, n, partials);
}

}  // namespace

int energy_grad_blocks() { return sm_count() * 4; }

void launch_grad_tables(const double* theta, const double* phi, int n, double* tab, cudaStream_t s) {
    k_grad_tables<<<(n + 127) / 128, 128, 0, s>>>(theta, phi, n, tab);
    note_launch();
}

void launch_energy_grad(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* pkey,
                        bool has_gen, double cos_t, double sin_t, const double* tab, int n, double* partials,
                        int blocks, cudaStream_t s) {
    switch (Wd) {
        case 1: launch_w<1>(rows, coef, M, pkey, has_gen, cos_t, sin_t, tab, n, partials, blocks, s); break;
        case 2: launch_w<2>(rows, coef, M, pkey, has_gen, cos_t, sin_t, tab, n, partials, blocks, s); break;
        default: launch_w<4>(rows, coef, M, pkey, has_gen, cos_t, sin_t, tab, n, partials, blocks, s); break;
    }
    note_launch();
}

}  // namespace iqcc
