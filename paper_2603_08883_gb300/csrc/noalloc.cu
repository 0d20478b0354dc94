// QMF energy without any device allocation.
//
// Some callers cannot allocate GPU memory at the moment they need an energy:
// a plug-in hosted by a framework that owns every byte of device memory
// through its own allocator, or a service that must keep a fixed memory
// footprint once started.  For them iqcc_qmf_energy_noalloc evaluates the same
// reduction as iqcc_qmf_energy (same kernels) on rows the caller already holds
// on the device, with its scratch - the per-block partial sums, the QMF
// product tables, the angles and the result - in the fixed array below, which
// every GPU that loads this library keeps until the process exits.
//
// The call copies the angles from host memory and reads the result back
// after synchronising its stream, so it cannot be recorded into a CUDA graph:
// on a stream that is being captured it returns IQCC_ERR_ARG before issuing
// any work, which leaves the caller's capture intact.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "iqcc_internal.cuh"

namespace iqcc {
void set_thread_error(const std::string& msg);  // abi.cu
}

using namespace iqcc;

namespace {

constexpr int kMaxBlocks = 4096;   // per-block partials of the energy pass
constexpr int kMaxQubits = 256;
constexpr int kMaxGroups = kMaxQubits / 4;
constexpr size_t kPartials = (size_t)kMaxBlocks * 3;
constexpr size_t kOut = 4;
constexpr size_t kAngles = 2 * kMaxQubits;
constexpr size_t kTables = (size_t)kMaxGroups * 256;
constexpr size_t kScratchDoubles = kPartials + kOut + kAngles + kTables;  // 233,988 bytes

// The scratch.  In host code this name is only a host-side stand-in for the
// device array: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_energy_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device (on the first call made with that device current).
cudaError_t scratch_on_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_energy_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

iqcc_status fail(iqcc_status st, const std::string& msg) {
    set_thread_error(msg);
    return st;
}

}  // namespace

extern "C" iqcc_status iqcc_qmf_energy_noalloc(int n_qubits, int64_t n_terms, const uint64_t* d_rows,
                                               const double* d_coef, const double* theta, const double* phi,
                                               void* stream, double* energy) {
    if (n_qubits < 1 || n_qubits > kMaxQubits)
        return fail(IQCC_ERR_ARG, "iqcc_qmf_energy_noalloc: n_qubits must be in 1..256 (the fixed scratch holds "
                                  "QMF tables for at most 256 qubits)");
    if (n_terms < 0) return fail(IQCC_ERR_ARG, "iqcc_qmf_energy_noalloc: n_terms < 0");
    if (n_terms > 0 && (!d_rows || !d_coef)) return fail(IQCC_ERR_ARG, "iqcc_qmf_energy_noalloc: null row array");
    if (!theta || !phi || !energy) return fail(IQCC_ERR_ARG, "iqcc_qmf_energy_noalloc: null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess)
        return fail(IQCC_ERR_CUDA, std::string("iqcc_qmf_energy_noalloc: cudaStreamIsCapturing: ") +
                                       cudaGetErrorString(e));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(IQCC_ERR_ARG, "iqcc_qmf_energy_noalloc: the stream is being captured; this call copies host "
                                  "arrays and synchronises its stream, so it cannot be recorded in a graph");
    const int blocks = expect_blocks();
    if (blocks > kMaxBlocks)
        return fail(IQCC_ERR_ARG, "iqcc_qmf_energy_noalloc: this GPU needs more partial sums than the fixed "
                                  "scratch holds (4096 blocks)");
    double* sc = nullptr;
    e = scratch_on_current_device(&sc);
    if (e != cudaSuccess)
        return fail(IQCC_ERR_CUDA, std::string("iqcc_qmf_energy_noalloc: cudaGetSymbolAddress: ") +
                                       cudaGetErrorString(e));
    double* partials = sc;
    double* out3 = partials + kPartials;
    double* angles = out3 + kOut;
    double* tables = angles + kAngles;

    const int n = n_qubits;
    const int Wd = device_words(n);
    const int groups = (n + 3) / 4;
    bool basis = true;
    uint64_t occ[4] = {0, 0, 0, 0};
    for (int j = 0; j < n; ++j) {
        if (theta[j] == 3.141592653589793) occ[j / 64] |= 1ull << (j % 64);
        else if (theta[j] != 0.0) basis = false;
    }
    if (!basis) {
        // every element the tables kernel reads is written here first
        if ((e = cudaMemcpyAsync(angles, theta, sizeof(double) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(angles + n, phi, sizeof(double) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return fail(IQCC_ERR_CUDA, std::string("iqcc_qmf_energy_noalloc: angle copy: ") + cudaGetErrorString(e));
        launch_qmf_tables(angles, angles + n, n, groups, tables, s);
    }
    const uint64_t zero_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // each block overwrites its own partials and the reduction overwrites out3:
    // nothing in the scratch has to start at zero
    launch_abc(Wd, d_rows, d_coef, n_terms, zero_key, basis, occ, tables, groups, partials, s);
    launch_reduce3(partials, blocks, out3, s);
    double h3[3];
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(h3, out3, sizeof h3, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(IQCC_ERR_CUDA, std::string("iqcc_qmf_energy_noalloc: ") + cudaGetErrorString(e));
    *energy = h3[0];
    return IQCC_OK;
}
