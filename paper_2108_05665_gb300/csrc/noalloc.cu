// Allocation-free linear XEB from device amplitudes.
//
// This is a variant of the plan's XEB reduction (kernels.cu: k_gather_xeb +
// k_xeb_final) for callers that cannot allocate device memory: processes whose
// device memory is owned by their own pool allocator (a cudaMalloc there fails
// or fights the pool), and latency-critical callers for whom the implicit
// device synchronisation of an allocation is not acceptable.  Its per-block
// partial sums live in the file-scope array below instead of in a workspace,
// so the entry point allocates nothing; the caller passes the amplitudes and
// the output buffer.
//
// The array is a device symbol: in host code its name is only a host-side
// stand-in, so the host obtains its device address once per device with
// cudaGetSymbolAddress (with that device current) and passes that address to
// the kernels.  Every device that loads this library holds the array
// (kNoAllocMaxBlocks x 2 doubles = 64 KiB) until the process exits.  All calls
// share it: calls whose kernels overlap on the GPU (different streams, or
// different host threads without ordering) race on it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "plan.h"
#include "xeb.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;                            // amplitudes per thread
constexpr int kPerBlock = kThreads * kPerThread;          // 4096
constexpr int kNoAllocMaxBlocks = 4096;
constexpr size_t kNoAllocMaxK = size_t(kNoAllocMaxBlocks) * kPerBlock;  // 16,777,216

// partial sums (sum p, sum p^2) of every block of the last call
static __device__ __align__(256) double g_xeb_scratch[2 * kNoAllocMaxBlocks];

std::mutex g_setup_mu;
double* g_scratch_ptr[64] = {nullptr};

__global__ void __launch_bounds__(kThreads) k_xeb_partials_noalloc(const double2* __restrict__ amps, int64_t k,
                                                                   double* __restrict__ scratch) {
    __shared__ double s1[kThreads], s2[kThreads];
    double a1 = 0.0, a2 = 0.0;
    const int64_t base = int64_t(blockIdx.x) * kPerBlock;
    for (int j = 0; j < kPerThread; ++j) {
        const int64_t i = base + int64_t(j) * kThreads + threadIdx.x;
        if (i < k) {
            const double2 a = amps[i];
            const double p = a.x * a.x + a.y * a.y;
            a1 += p;
            a2 += p * p;
        }
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int d = kThreads / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) {
            s1[threadIdx.x] += s1[threadIdx.x + d];
            s2[threadIdx.x] += s2[threadIdx.x + d];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {  // every block writes its own slot: nothing needs clearing
        scratch[2 * blockIdx.x] = s1[0];
        scratch[2 * blockIdx.x + 1] = s2[0];
    }
}

__global__ void __launch_bounds__(kThreads) k_xeb_final_noalloc(const double* __restrict__ scratch, int nb,
                                                                int64_t k, int n, double* __restrict__ out) {
    __shared__ double s1[kThreads], s2[kThreads];
    double a1 = 0.0, a2 = 0.0;
    for (int b = threadIdx.x; b < nb; b += kThreads) {
        a1 += scratch[2 * b];
        a2 += scratch[2 * b + 1];
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int d = kThreads / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) {
            s1[threadIdx.x] += s1[threadIdx.x + d];
            s2[threadIdx.x] += s2[threadIdx.x + d];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double scale = ldexp(1.0, n);
        const double mean = scale * s1[0] / double(k);
        out[0] = mean - 1.0;
        out[1] = mean;
        out[2] = scale * scale * s2[0] / double(k);
    }
}

xeb_status fail(xeb_status s, const std::string& m) {
    xebp::set_last_error(m);
    return s;
}

}  // namespace

extern "C" xeb_status xeb_linear_xeb_noalloc(const double* amps_dev, size_t k, int n_qubits, double* out_dev,
                                             uintptr_t stream) {
    if (!amps_dev || !out_dev) return fail(XEB_EINVAL, "amplitude and output pointers must be device pointers");
    if (reinterpret_cast<uintptr_t>(amps_dev) % 16 != 0)
        return fail(XEB_EINVAL, "amps_dev must be 16-byte aligned (amplitudes are read as 16-byte complex values)");
    if (k == 0) return fail(XEB_EINVAL, "need k >= 1 amplitudes");
    if (k > kNoAllocMaxK)
        return fail(XEB_EINVAL, "k = " + std::to_string(k) + " exceeds the allocation-free limit of " +
                                    std::to_string(kNoAllocMaxK) + " amplitudes (fixed scratch of " +
                                    std::to_string(kNoAllocMaxBlocks) + " block partials)");
    if (n_qubits < 1 || n_qubits > 64) return fail(XEB_EINVAL, "n_qubits must be in [1, 64]");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(XEB_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(XEB_EUNSUPPORTED, "device index beyond 63");
    double* scratch = nullptr;
    {
        // first call on this device: resolve the device address of the
        // scratch symbol (the device is current here)
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_xeb_scratch);
            if (e != cudaSuccess || !p)
                return fail(XEB_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nb = int((k + kPerBlock - 1) / kPerBlock);
    k_xeb_partials_noalloc<<<nb, kThreads, 0, st>>>(reinterpret_cast<const double2*>(amps_dev), int64_t(k), scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(XEB_ECUDA, std::string("partials launch: ") + cudaGetErrorString(e));
    k_xeb_final_noalloc<<<1, kThreads, 0, st>>>(scratch, nb, int64_t(k), n_qubits, out_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(XEB_ECUDA, std::string("final launch: ") + cudaGetErrorString(e));
    return XEB_OK;
}
