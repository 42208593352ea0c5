// Allocation-free variant of the diagnostic integrals (mass, momenta and
// total entropy) for callers that cannot call cudaMalloc: code that runs
// while another runtime owns the device memory pool (a host framework's
// caching allocator that must see every allocation), real-time loops in which
// the implicit device synchronisation of cudaMalloc/cudaFree is not
// acceptable, and embedded hosts with a fixed memory budget decided at start
// up. The caller passes every input and the output; the per-element partial
// sums live in a fixed, file-scope device array of this library.
#include <mutex>
#include <string>

#include "kcommon.cuh"

namespace swe {
namespace {

constexpr int kNoAllocMaxElements = SWE_NOALLOC_MAX_ELEMENTS;
constexpr int kMaxDevices = 64;

// Four partial sums per element (sum of w J h, w J hu, w J hv, w J e): 2 MiB.
// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_partials[4 * kNoAllocMaxElements];

// Device address of g_partials per device, resolved once per device.
double* g_addr[kMaxDevices] = {};
std::mutex g_mu;

// One warp per element: the element's four sums in a fixed order (lane
// partials, then a butterfly), written to partials[c * K + k]. Every slot the
// second pass reads is written here first, so nothing needs clearing.
__global__ void k_element_integrals(int nn, int K, const double* __restrict__ W,
                                    const double* __restrict__ wJ, const double* __restrict__ b,
                                    double g, double* __restrict__ partials) {
    const int lane = threadIdx.x & 31;
    const long long k = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= K) return;
    const long long KN = (long long)K * nn;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int node = lane; node < nn; node += 32) {
        const long long id = k * nn + node;
        const double w = wJ[id], h = W[id], hu = W[KN + id], hv = W[2 * KN + id];
        s0 = fma(w, h, s0);
        s1 = fma(w, hu, s1);
        s2 = fma(w, hv, s2);
        const double kin = h > 0.0 ? 0.5 * fma(hu, hu, hv * hv) / h : 0.0;
        s3 = fma(w, kin + g * h * fma(0.5, h, b[id]), s3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    }
    if (lane == 0) {
        partials[k] = s0;
        partials[K + k] = s1;
        partials[2 * (long long)K + k] = s2;
        partials[3 * (long long)K + k] = s3;
    }
}

// One block of 4 warps, warp c sums component c over the K element partials
// in a fixed order and writes out[c].
__global__ void k_sum_integrals(int K, const double* __restrict__ partials, double* __restrict__ out) {
    const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
    double s = 0.0;
    for (int k = lane; k < K; k += 32) s += partials[(long long)c * K + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[c] = s;
}

int nfail(const std::string& m) { return set_last_error(SWE_ERR_ARG, m); }

// 0 if p is device (or managed) memory that the current device `dev` can
// use directly; an error code (with the message set) otherwise. A pointer of
// another device would make the kernels read across devices or fault.
int check_pointer(const void* p, const char* name, int dev) {
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();  // the failed query sets the (non-sticky) last error: clear it
        return nfail(std::string("swe_integrals_noalloc: ") + name + " is not a CUDA allocation");
    }
    if (a.type == cudaMemoryTypeManaged) return SWE_OK;
    if (a.type != cudaMemoryTypeDevice)
        return nfail(std::string("swe_integrals_noalloc: ") + name + " is not device memory");
    if (a.device != dev)
        return nfail(std::string("swe_integrals_noalloc: ") + name + " is on device " + std::to_string(a.device) +
                     ", the current device is " + std::to_string(dev));
    return SWE_OK;
}

}  // namespace
}  // namespace swe

extern "C" int swe_integrals_noalloc(int N, int K, const double* W, const double* wJ, const double* b,
                                     double g, double* out4, void* stream) {
    using namespace swe;
    if (N < 1 || N > NMAX) return nfail("swe_integrals_noalloc: N must be in 1..12");
    if (K < 1) return nfail("swe_integrals_noalloc: K must be >= 1");
    if (K > kNoAllocMaxElements)
        return nfail("swe_integrals_noalloc: K = " + std::to_string(K) + " exceeds the fixed scratch limit of " +
                     std::to_string(kNoAllocMaxElements) + " elements");
    if (!W || !wJ || !b || !out4) return nfail("swe_integrals_noalloc: NULL pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        return set_last_error(SWE_ERR_CUDA, std::string("swe_integrals_noalloc: cudaGetDevice: ") +
                                                cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= kMaxDevices) return nfail("swe_integrals_noalloc: device index out of range");
    {
        const void* ptrs[4] = {W, wJ, b, out4};
        const char* names[4] = {"W", "wJ", "b", "out4"};
        for (int i = 0; i < 4; ++i) {
            int rc = check_pointer(ptrs[i], names[i], dev);
            if (rc != SWE_OK) return rc;
        }
    }
    double* scratch = nullptr;
    {
        // First call on each device: resolve the device address of the
        // array with that device current (host code must not use the symbol
        // itself, which is only a host-side stand-in).
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_partials);
            if (e != cudaSuccess || !p) {
                return set_last_error(SWE_ERR_CUDA, std::string("swe_integrals_noalloc: cudaGetSymbolAddress: ") +
                                                        cudaGetErrorString(e));
            }
            g_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_addr[dev];
    }
    const int nn = (N + 1) * (N + 1);
    cudaStream_t s = (cudaStream_t)stream;
    constexpr int WPB = 4;
    k_element_integrals<<<(K + WPB - 1) / WPB, 32 * WPB, 0, s>>>(nn, K, W, wJ, b, g, scratch);
    k_sum_integrals<<<1, 128, 0, s>>>(K, scratch, out4);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        return set_last_error(SWE_ERR_CUDA, std::string("swe_integrals_noalloc: launch: ") + cudaGetErrorString(e));
    }
    return SWE_OK;
}
