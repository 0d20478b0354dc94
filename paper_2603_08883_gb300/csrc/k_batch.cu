// Many independent Hamiltonians in one context (uneven sizes, up to 48 qubits
// each, one 64-bit word per x and z).  Problem b's strings carry b in bits
// 48..63 of their z word: Z letters on virtual qubits that no generator or
// candidate touches, so they cancel in every product inside a problem, keep
// the keys of different problems apart in every index and sort, and add a
// factor <Z> = 1 (theta = 0 there) to every expectation.  These kernels are
// the per-problem reductions of the path for z-eigenstate references (every
// theta_j 0 or pi, the reference of the batch workloads): the energy (Eq. 12
// at tau = 0), DIS screening (Eq. 14-15) down to each problem's best
// candidate, and the closed-form A, B, C and tau* of that candidate.
#include <cuda_runtime.h>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kThreads = 256;
constexpr uint64_t kXMask = (1ull << kBatchTagShift) - 1;

__device__ __forceinline__ int tag_of(uint64_t z) { return (int)(z >> kBatchTagShift); }

__device__ __forceinline__ uint64_t abs_bits_g(double c) {
    return (uint64_t)__double_as_longlong(c) & 0x7FFFFFFFFFFFFFFFull;
}

// <T> on a z-eigenstate with occupation occ: (-1)^{popc(z & occ)} when x = 0, else 0.
__device__ __forceinline__ double basis_value(uint64_t x, uint64_t z, uint64_t occ) {
    if (x & kXMask) return 0.0;
    return (__popcll(z & occ) & 1) ? -1.0 : 1.0;
}

// Per-problem energy and term count: acc[b], cnt[b] per block, B <= kMaxBatch.
__global__ void __launch_bounds__(kThreads) k_seg_energy(const uint64_t* __restrict__ rows,
                                                         const double* __restrict__ coef, int64_t M,
                                                         const uint64_t* __restrict__ occ, int B, double* partials,
                                                         unsigned long long* counts) {
    extern __shared__ double sm[];
    double* acc = sm;
    unsigned int* cnt = reinterpret_cast<unsigned int*>(sm + B);
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        acc[b] = 0.0;
        cnt[b] = 0u;
    }
    __syncthreads();
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += s) {
        const uint64_t x = rows[2 * i], z = rows[2 * i + 1];
        const int b = tag_of(z);
        if (b >= B) continue;
        atomicAdd(cnt + b, 1u);
        const double v = basis_value(x, z, occ[b]);
        if (v != 0.0) atomicAdd(acc + b, v * coef[i]);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        partials[(size_t)blockIdx.x * B + b] = acc[b];
        if (cnt[b]) atomicAdd(counts + b, (unsigned long long)cnt[b]);
    }
}

// DIS groups keyed by (flip set, problem): key = x | tag, stored in the slot
// itself (a single 64-bit CAS publishes it; keys stay below 2^60, never the
// empty pattern), with the group's gradient summed in gsum[slot].  A row T with
// flip set F = x_T != 0 adds s C_T <Q> for alpha = (x = F, z = lowest bit of F)
// when T anticommutes with alpha (Q = T xor alpha is diagonal: Eq. 15).
__global__ void __launch_bounds__(kThreads) k_seg_dis_group(const uint64_t* __restrict__ rows,
                                                            const double* __restrict__ coef, int64_t M,
                                                            const uint64_t* __restrict__ occ, int B, uint64_t* slots,
                                                            double* gsum, uint64_t bucket_mask, int max_probe,
                                                            DevCounters* ctr) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += s) {
        const uint64_t x = rows[2 * i], z = rows[2 * i + 1];
        const uint64_t f = x & kXMask;
        const int b = tag_of(z);
        if (!f || b >= B) continue;
        const uint64_t key = f | ((uint64_t)b << kBatchTagShift);
        Key<1> kk;
        kk.x[0] = key;
        kk.z[0] = 0;
        uint64_t bk = hash_key<1>(kk) & bucket_mask;
        int64_t slot = -1;
        for (int p = 0; p < max_probe && slot < 0; ++p) {
            for (int t = 0; t < 4 && slot < 0; ++t) {
                unsigned long long* sl = reinterpret_cast<unsigned long long*>(slots + bk * 4 + t);
                unsigned long long cur = *(volatile unsigned long long*)sl;
                if (cur == kEmptySlot) cur = atomicCAS(sl, (unsigned long long)kEmptySlot, (unsigned long long)key);
                if (cur == kEmptySlot || cur == key) slot = (int64_t)(bk * 4 + t);
            }
            bk = (bk + 1) & bucket_mask;
        }
        if (slot < 0) {
            set_error(ctr, IQCC_ERR_HASH_FULL, 50);
            continue;
        }
        Key<1> t;
        t.x[0] = x;
        t.z[0] = z;
        Key<1> a;
        a.x[0] = f;
        a.z[0] = f & (~f + 1);
        if (!anticommutes<1>(t, a)) continue;
        const Key<1> q = key_xor<1>(t, a);
        const int sg = product_sign<1>(t, 1, a, q);
        const bool neg = (sg < 0) ^ ((__popcll(q.z[0] & occ[b]) & 1) != 0);
        atomicAdd(gsum + slot, neg ? -coef[i] : coef[i]);
    }
}

// Best candidate per problem: largest |g| with its 20 low mantissa bits
// cleared, ties to the smaller key (the canonical order of the candidates).
__global__ void k_seg_best_coarse(const uint64_t* __restrict__ slots, const double* __restrict__ gsum, uint64_t n_slots,
                                  int B, unsigned long long* best_coarse) {
    const uint64_t s = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += s) {
        const uint64_t key = slots[i];
        if (key == kEmptySlot) continue;
        const int b = (int)(key >> kBatchTagShift);
        if (b < B) atomicMax(best_coarse + b, (unsigned long long)(abs_bits_g(gsum[i]) & ~0xFFFFFull));
    }
}

__global__ void k_seg_best_key(const uint64_t* __restrict__ slots, const double* __restrict__ gsum, uint64_t n_slots,
                               int B, const unsigned long long* __restrict__ best_coarse,
                               unsigned long long* best_key) {
    const uint64_t s = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += s) {
        const uint64_t key = slots[i];
        if (key == kEmptySlot) continue;
        const int b = (int)(key >> kBatchTagShift);
        if (b < B && (abs_bits_g(gsum[i]) & ~0xFFFFFull) == best_coarse[b]) atomicMin(best_key + b, key);
    }
}

__global__ void k_seg_best_grad(const uint64_t* __restrict__ slots, const double* __restrict__ gsum, uint64_t n_slots,
                                int B, const unsigned long long* __restrict__ best_key, double* best_g) {
    const uint64_t s = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += s) {
        const uint64_t key = slots[i];
        if (key == kEmptySlot) continue;
        const int b = (int)(key >> kBatchTagShift);
        if (b < B && key == best_key[b]) best_g[b] = gsum[i];
    }
}

// A, B, C of each problem's best candidate (none: everything in A).
__global__ void __launch_bounds__(kThreads) k_seg_abc(const uint64_t* __restrict__ rows,
                                                      const double* __restrict__ coef, int64_t M,
                                                      const uint64_t* __restrict__ occ, int B,
                                                      const unsigned long long* __restrict__ best_key,
                                                      double* partials) {
    extern __shared__ double sm[];
    for (int k = threadIdx.x; k < 3 * B; k += blockDim.x) sm[k] = 0.0;
    __syncthreads();
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += s) {
        const uint64_t x = rows[2 * i], z = rows[2 * i + 1];
        const int b = tag_of(z);
        if (b >= B) continue;
        const double c = coef[i];
        const uint64_t bk = best_key[b];
        Key<1> t;
        t.x[0] = x;
        t.z[0] = z;
        Key<1> a;
        a.x[0] = bk == kEmptySlot ? 0ull : (bk & kXMask);
        a.z[0] = a.x[0] & (~a.x[0] + 1);
        if (!anticommutes<1>(t, a)) {
            const double v = basis_value(x, z, occ[b]);
            if (v != 0.0) atomicAdd(sm + 3 * b, v * c);
            continue;
        }
        const double vt = basis_value(x, z, occ[b]);
        if (vt != 0.0) atomicAdd(sm + 3 * b + 1, vt * c);
        const Key<1> q = key_xor<1>(t, a);
        const double vq = basis_value(q.x[0], q.z[0], occ[b]);
        if (vq != 0.0) atomicAdd(sm + 3 * b + 2, (double)product_sign<1>(t, 1, a, q) * vq * c);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * B; k += blockDim.x) partials[(size_t)blockIdx.x * 3 * B + k] = sm[k];
}

// tau* = atan2(-C, -B) (0 when B = C = 0) and the generator of each problem's dress.
__global__ void k_seg_tau(const double* __restrict__ abc, const unsigned long long* __restrict__ best_key, int B,
                          double* tau, Gen<1>* gens) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double bb = abc[3 * b + 1], cc = abc[3 * b + 2];
    const uint64_t bk = best_key[b];
    const bool none = bk == kEmptySlot;
    const double t = (none || (bb == 0.0 && cc == 0.0)) ? 0.0 : atan2(-cc, -bb);
    tau[b] = t;
    Gen<1> g{};
    g.p.x[0] = none ? 0ull : (bk & kXMask);
    g.p.z[0] = g.p.x[0] & (~g.p.x[0] + 1);  // single Y on the lowest flipped qubit
    g.yP = __popcll(g.p.x[0] & g.p.z[0]) & 3;
    g.top_word = 0;
    g.top_mask = g.p.z[0];                  // lowest set bit of the first non-zero word (x)
    g.cos_t = cos(t);
    g.sin_t = sin(t);
    gens[b] = g;
}

}  // namespace

void launch_seg_energy(const uint64_t* rows, const double* coef, int64_t M, const uint64_t* occ, int B,
                       double* partials, unsigned long long* counts, int blocks, cudaStream_t s) {
    const size_t smem = (size_t)B * (sizeof(double) + sizeof(unsigned int));
    k_seg_energy<<<blocks, kThreads, smem, s>>>(rows, coef, M, occ, B, partials, counts);
    note_launch();
}

void launch_seg_dis_group(const uint64_t* rows, const double* coef, int64_t M, const uint64_t* occ, int B,
                          uint64_t* slots, double* gsum, uint64_t bucket_mask, int max_probe, DevCounters* ctr,
                          int blocks, cudaStream_t s) {
    k_seg_dis_group<<<blocks, kThreads, 0, s>>>(rows, coef, M, occ, B, slots, gsum, bucket_mask, max_probe, ctr);
    note_launch();
}

void launch_seg_best(const uint64_t* slots, const double* gsum, uint64_t n_slots, int B,
                     unsigned long long* best_coarse, unsigned long long* best_key, double* best_g, int blocks,
                     cudaStream_t s) {
    k_seg_best_coarse<<<blocks, kThreads, 0, s>>>(slots, gsum, n_slots, B, best_coarse);
    k_seg_best_key<<<blocks, kThreads, 0, s>>>(slots, gsum, n_slots, B, best_coarse, best_key);
    k_seg_best_grad<<<blocks, kThreads, 0, s>>>(slots, gsum, n_slots, B, best_key, best_g);
    note_launch(3);
}

void launch_seg_abc(const uint64_t* rows, const double* coef, int64_t M, const uint64_t* occ, int B,
                    const unsigned long long* best_key, double* partials, int blocks, cudaStream_t s) {
    k_seg_abc<<<blocks, kThreads, (size_t)3 * B * sizeof(double), s>>>(rows, coef, M, occ, B, best_key, partials);
    note_launch();
}

void launch_seg_tau(const double* abc, const unsigned long long* best_key, int B, double* tau, Gen<1>* gens,
                    cudaStream_t s) {
    k_seg_tau<<<(B + 127) / 128, 128, 0, s>>>(abc, best_key, B, tau, gens);
    note_launch();
}

}  // namespace iqcc
