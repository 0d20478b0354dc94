// Learned term screening: a perceptron scores every term of H, and the term
// limit keeps the highest scores instead of the largest |C|.
//
// Features of a term T with coefficient C (kFeat of them, in FP32, from its key;
// G = union of the supports of the iteration's generators, <T> at the
// reference product state of Eq. 3):
//   0  log10|C| / 8           1  min(flipped qubits, 16) / 16
//   2  min(Y letters, 16) / 16                           3  Z letters on G / 8
//   4  |supp T & G| / 8        5  |flips & G| / 8        6  <T>
//   7  1 when every flip of T lies in G (and T has one)
// None grows with the number of qubits: the counts that could (flips, Y
// letters) saturate, and Z letters count only on G (a Z off G neither changes
// whether T commutes with a generator nor |<T>| at a basis reference).
// Model: 8 -> 256 -> 256 -> 1 with ReLU, BF16 weights and activations, FP32
// accumulation, on the tensor cores (mma.sync m16n8k16).  One warp scores 16
// terms at a time: layer 1 is one MMA per 8 hidden units; its accumulator
// fragments for two adjacent groups of 8 units are exactly the A fragment of
// one 16-wide K step of layer 2, so the hidden activations never leave
// registers; layer 3 is folded into layer 2's epilogue (ReLU, times w3, summed
// across the 4 lanes that share a row).  Layer-2 weights sit in shared memory
// with rows padded to 264 elements so that the 8 rows a fragment load touches
// fall in distinct banks.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "iqcc_internal.cuh"

namespace iqcc {

namespace {

constexpr int kFeat = 8;
constexpr int kHid = 256;
constexpr int kW1Stride = 24;   // bf16 per layer-1 row in shared memory (16 used)
constexpr int kW2Stride = 264;  // bf16 per layer-2 row in shared memory (256 used)
constexpr int kMlpThreads = 384;
constexpr int kMlpWarps = kMlpThreads / 32;
// Layer-2 output tiles of 8 computed together (8e8 terms: 1 tile 304 ms, 2 tiles
// 268 ms, 4 tiles 263 ms).
constexpr int kL2Tiles = 4;

// Device model layout (bytes): w1 [256][16] bf16 (inputs 8..15 zero), w2
// [256][256] bf16 (row = output unit), then float b1[256], b2[256], w3[256], b3.
constexpr size_t kOffW1 = 0;
constexpr size_t kOffW2 = kOffW1 + (size_t)kHid * 16 * 2;
constexpr size_t kOffB1 = kOffW2 + (size_t)kHid * kHid * 2;
constexpr size_t kOffB2 = kOffB1 + kHid * 4;
constexpr size_t kOffW3 = kOffB2 + kHid * 4;
constexpr size_t kOffB3 = kOffW3 + kHid * 4;
constexpr size_t kModelBytes = kOffB3 + 16;

template <int W>
struct GenSupport {
    uint64_t g[W];  // union of the generators' supports
};

// log10|c| in FP32 from the double's exponent and a float log of its mantissa
// (no FP64 transcendental: GB300's FP64 rate is low); -300 for c = 0.
__device__ __forceinline__ float log10_abs(double c) {
    if (c == 0.0) return -300.0f;
    int e;
    const double m = frexp(fabs(c), &e);  // |c| = m 2^e, m in [0.5, 1)
    return (log2f((float)m) + (float)e) * 0.30102999566f;
}

// ev: per-qubit <I>, <X>, <Y>, <Z> as floats (4 per qubit).
template <int W>
__device__ __forceinline__ void term_features(const Key<W>& t, double c, const GenSupport<W>& gs, const float* ev,
                                              float* f) {
    int flips = 0, ys = 0, zg = 0, ov = 0, fov = 0;
    float e = 1.0f;
#pragma unroll
    for (int wd = 0; wd < W; ++wd) {
        const uint64_t x = t.x[wd], z = t.z[wd];
        flips += __popcll(x);
        ys += __popcll(x & z);
        zg += __popcll(z & ~x & gs.g[wd]);
        ov += __popcll((x | z) & gs.g[wd]);
        fov += __popcll(x & gs.g[wd]);
        uint64_t m = x | z;
        while (m && e != 0.0f) {
            const int j = __ffsll((long long)m) - 1;
            m &= m - 1;
            const int xb = (int)((x >> j) & 1ull), zb = (int)((z >> j) & 1ull);
            e *= ev[4 * (64 * wd + j) + (xb ? (zb ? 2 : 1) : 3)];
        }
    }
    f[0] = log10_abs(c) / 8.0f;
    f[1] = min(flips, 16) / 16.0f;
    f[2] = min(ys, 16) / 16.0f;
    f[3] = zg / 8.0f;
    f[4] = ov / 8.0f;
    f[5] = fov / 8.0f;
    f[6] = e;
    f[7] = (flips > 0 && fov == flips) ? 1.0f : 0.0f;
}

// The per-qubit <sigma> of the double table (stride ts, letters at 0..3) as floats.
__device__ __forceinline__ void load_ev(const double* ev_g, int ts, int n, float* ev) {
    for (int i = threadIdx.x; i < 4 * n; i += blockDim.x) ev[i] = (float)ev_g[ts * (i / 4) + (i % 4)];
}

template <int W>
__global__ void k_term_features(const uint64_t* __restrict__ rows, const double* __restrict__ coef, int64_t M,
                                GenSupport<W> gs, const double* __restrict__ ev_g, int ts, int n, float* out) {
    extern __shared__ float evf[];
    load_ev(ev_g, ts, n, evf);
    __syncthreads();
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += s) {
        float f[kFeat];
        term_features<W>(load_key<W>(rows, i), coef[i], gs, evf, f);
#pragma unroll
        for (int k = 0; k < kFeat; ++k) out[(size_t)i * kFeat + k] = f[k];
    }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The term limit's key: a positive double increasing with the score (exact:
// a float plus 1024 is representable), scores below -1000 all at 24.
__device__ __forceinline__ double rank_of(float score) { return (double)fmaxf(score, -1000.0f) + 1024.0; }

// score[i] (may be NULL) and rank[i] = rank_of(score) (the term limit's key).
template <int W>
__global__ void __launch_bounds__(kMlpThreads, 1) k_mlp_score(const uint64_t* __restrict__ rows,
                                                              const double* __restrict__ coef, int64_t M,
                                                              GenSupport<W> gs, const double* __restrict__ ev_g,
                                                              int ts, int n, const unsigned char* __restrict__ model,
                                                              float* score, double* rank) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* w1 = reinterpret_cast<__nv_bfloat16*>(smem_raw);           // [256][24]
    __nv_bfloat16* w2 = w1 + kHid * kW1Stride;                                 // [256][264]
    float* b1 = reinterpret_cast<float*>(w2 + kHid * kW2Stride);
    float* b2 = b1 + kHid;
    float* w3 = b2 + kHid;
    float* stage = w3 + kHid;                                                  // [warps][16][16]
    float* ev = stage + kMlpWarps * 256;                                       // [4 n]
    const __nv_bfloat16* mw1 = reinterpret_cast<const __nv_bfloat16*>(model + kOffW1);
    const __nv_bfloat16* mw2 = reinterpret_cast<const __nv_bfloat16*>(model + kOffW2);
    for (int i = threadIdx.x; i < kHid * 16; i += blockDim.x) w1[(i / 16) * kW1Stride + (i % 16)] = mw1[i];
    for (int i = threadIdx.x; i < kHid * kHid / 8; i += blockDim.x) {  // 16-byte chunks
        const int r = i / (kHid / 8), cc = i % (kHid / 8);
        *reinterpret_cast<uint4*>(w2 + r * kW2Stride + 8 * cc) = reinterpret_cast<const uint4*>(mw2)[i];
    }
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
        b1[i] = reinterpret_cast<const float*>(model + kOffB1)[i];
        b2[i] = reinterpret_cast<const float*>(model + kOffB2)[i];
        w3[i] = reinterpret_cast<const float*>(model + kOffW3)[i];
    }
    load_ev(ev_g, ts, n, ev);
    const float b3 = *reinterpret_cast<const float*>(model + kOffB3);
    __syncthreads();

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    float* st = stage + wid * 256;
    const int64_t n_tiles = (M + 15) / 16;
    const int64_t warps = (int64_t)gridDim.x * kMlpWarps;
    for (int64_t tile = (int64_t)blockIdx.x * kMlpWarps + wid; tile < n_tiles; tile += warps) {
        // features of the tile's 16 terms (lanes 0..15), zero rows past M
        if (lane < 16) {
            const int64_t i = tile * 16 + lane;
            float f[kFeat];
            if (i < M) {
                term_features<W>(load_key<W>(rows, i), coef[i], gs, ev, f);
            } else {
#pragma unroll
                for (int k = 0; k < kFeat; ++k) f[k] = 0.0f;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) st[lane * 16 + k] = k < kFeat ? f[k] : 0.0f;
        }
        __syncwarp();
        uint32_t a1[4];
        a1[0] = pack_bf16(st[g * 16 + 2 * t], st[g * 16 + 2 * t + 1]);
        a1[1] = pack_bf16(st[(g + 8) * 16 + 2 * t], st[(g + 8) * 16 + 2 * t + 1]);
        a1[2] = pack_bf16(st[g * 16 + 2 * t + 8], st[g * 16 + 2 * t + 9]);
        a1[3] = pack_bf16(st[(g + 8) * 16 + 2 * t + 8], st[(g + 8) * 16 + 2 * t + 9]);
        // layer 1 -> A fragments of layer 2
        uint32_t h[16][4];
#pragma unroll
        for (int jn = 0; jn < kHid / 8; ++jn) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            const __nv_bfloat16* wr = w1 + (8 * jn + g) * kW1Stride;
            mma_bf16(c, a1, *reinterpret_cast<const uint32_t*>(wr + 2 * t),
                     *reinterpret_cast<const uint32_t*>(wr + 2 * t + 8));
            const int n0 = 8 * jn + 2 * t;
            const float v0 = fmaxf(c[0] + b1[n0], 0.f), v1 = fmaxf(c[1] + b1[n0 + 1], 0.f);
            const float v2 = fmaxf(c[2] + b1[n0], 0.f), v3 = fmaxf(c[3] + b1[n0 + 1], 0.f);
            h[jn >> 1][(jn & 1) * 2] = pack_bf16(v0, v1);
            h[jn >> 1][(jn & 1) * 2 + 1] = pack_bf16(v2, v3);
        }
        // layer 2, with layer 3 in the epilogue; kL2Tiles independent accumulators
        // per step so that consecutive MMAs do not wait on each other
        float s_lo = 0.f, s_hi = 0.f;
#pragma unroll 1
        for (int jn0 = 0; jn0 < kHid / 8; jn0 += kL2Tiles) {
            float c[kL2Tiles][4];
#pragma unroll
            for (int u = 0; u < kL2Tiles; ++u) c[u][0] = c[u][1] = c[u][2] = c[u][3] = 0.f;
#pragma unroll
            for (int kk = 0; kk < kHid / 16; ++kk) {
#pragma unroll
                for (int u = 0; u < kL2Tiles; ++u) {
                    const __nv_bfloat16* wr = w2 + (8 * (jn0 + u) + g) * kW2Stride + 16 * kk + 2 * t;
                    mma_bf16(c[u], h[kk], *reinterpret_cast<const uint32_t*>(wr),
                             *reinterpret_cast<const uint32_t*>(wr + 8));
                }
            }
#pragma unroll
            for (int u = 0; u < kL2Tiles; ++u) {
                const int n0 = 8 * (jn0 + u) + 2 * t;
                s_lo += fmaxf(c[u][0] + b2[n0], 0.f) * w3[n0] + fmaxf(c[u][1] + b2[n0 + 1], 0.f) * w3[n0 + 1];
                s_hi += fmaxf(c[u][2] + b2[n0], 0.f) * w3[n0] + fmaxf(c[u][3] + b2[n0 + 1], 0.f) * w3[n0 + 1];
            }
        }
        s_lo += __shfl_xor_sync(0xFFFFFFFFu, s_lo, 1);
        s_lo += __shfl_xor_sync(0xFFFFFFFFu, s_lo, 2);
        s_hi += __shfl_xor_sync(0xFFFFFFFFu, s_hi, 1);
        s_hi += __shfl_xor_sync(0xFFFFFFFFu, s_hi, 2);
        if (t == 0) {
            const int64_t i0 = tile * 16 + g, i1 = i0 + 8;
            if (i0 < M) {
                if (score) score[i0] = s_lo + b3;
                rank[i0] = rank_of(s_lo + b3);
            }
            if (i1 < M) {
                if (score) score[i1] = s_hi + b3;
                rank[i1] = rank_of(s_hi + b3);
            }
        }
        __syncwarp();
    }
}

template <int W>
GenSupport<W> support_of(const uint64_t* gsup) {
    GenSupport<W> s{};
    for (int j = 0; j < W; ++j) s.g[j] = gsup[j];
    return s;
}

size_t mlp_smem(int ts, int n) {
    return (size_t)kHid * kW1Stride * 2 + (size_t)kHid * kW2Stride * 2 + 3 * kHid * 4 + kMlpWarps * 256 * 4 +
           (size_t)4 * n * 4;
}

__global__ void k_gather_words(const uint32_t* __restrict__ in, const uint32_t* __restrict__ perm, int64_t n, int words,
                               uint32_t* out) {
    const int64_t s = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n * words; k += s) {
        const int64_t i = k / words;
        out[k] = in[(int64_t)perm[i] * words + (k - i * words)];
    }
}

}  // namespace

void launch_gather_bytes(const void* in, const uint32_t* perm, int64_t n, int width, void* out, cudaStream_t s) {
    if (n <= 0) return;
    k_gather_words<<<sm_count() * 4, 256, 0, s>>>((const uint32_t*)in, perm, n, width / 4, (uint32_t*)out);
    note_launch();
}

int screen_features() { return kFeat; }
size_t screen_model_bytes() { return kModelBytes; }

void launch_term_features(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* gsup,
                          const double* ev, int ts, int n, float* out, cudaStream_t s) {
    if (M <= 0) return;
    const int grid = sm_count() * 4;
    const size_t smem = (size_t)4 * n * 4;
    switch (Wd) {
        case 1: k_term_features<1><<<grid, 256, smem, s>>>(rows, coef, M, support_of<1>(gsup), ev, ts, n, out); break;
        case 2: k_term_features<2><<<grid, 256, smem, s>>>(rows, coef, M, support_of<2>(gsup), ev, ts, n, out); break;
        default: k_term_features<4><<<grid, 256, smem, s>>>(rows, coef, M, support_of<4>(gsup), ev, ts, n, out); break;
    }
    note_launch();
}

void launch_mlp_score(int Wd, const uint64_t* rows, const double* coef, int64_t M, const uint64_t* gsup,
                      const double* ev, int ts, int n, const void* model, float* score, double* rank,
                      cudaStream_t s) {
    if (M <= 0) return;
    const size_t smem = mlp_smem(ts, n);
    const int grid = sm_count();
    const unsigned char* m = (const unsigned char*)model;
    switch (Wd) {
        case 1:
            cudaFuncSetAttribute(k_mlp_score<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_mlp_score<1><<<grid, kMlpThreads, smem, s>>>(rows, coef, M, support_of<1>(gsup), ev, ts, n, m, score, rank);
            break;
        case 2:
            cudaFuncSetAttribute(k_mlp_score<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_mlp_score<2><<<grid, kMlpThreads, smem, s>>>(rows, coef, M, support_of<2>(gsup), ev, ts, n, m, score, rank);
            break;
        default:
            cudaFuncSetAttribute(k_mlp_score<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_mlp_score<4><<<grid, kMlpThreads, smem, s>>>(rows, coef, M, support_of<4>(gsup), ev, ts, n, m, score, rank);
            break;
    }
    note_launch();
}

// Host float weights -> the device layout (bf16 conversion on the host side of the copy).
void pack_screen_model(const float* w1, const float* b1, const float* w2, const float* b2, const float* w3, float b3,
                       unsigned char* out) {
    __nv_bfloat16* ow1 = reinterpret_cast<__nv_bfloat16*>(out + kOffW1);
    __nv_bfloat16* ow2 = reinterpret_cast<__nv_bfloat16*>(out + kOffW2);
    for (int r = 0; r < kHid; ++r)
        for (int k = 0; k < 16; ++k) ow1[r * 16 + k] = __float2bfloat16_rn(k < kFeat ? w1[r * kFeat + k] : 0.0f);
    for (int i = 0; i < kHid * kHid; ++i) ow2[i] = __float2bfloat16_rn(w2[i]);
    float* ob1 = reinterpret_cast<float*>(out + kOffB1);
    float* ob2 = reinterpret_cast<float*>(out + kOffB2);
    float* ow3 = reinterpret_cast<float*>(out + kOffW3);
    for (int i = 0; i < kHid; ++i) {
        ob1[i] = b1[i];
        ob2[i] = b2[i];
        ow3[i] = w3[i];
    }
    *reinterpret_cast<float*>(out + kOffB3) = b3;
}

}  // namespace iqcc
