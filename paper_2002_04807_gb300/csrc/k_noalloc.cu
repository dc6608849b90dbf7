// Allocation-free variant of the Rayleigh-Ritz Gram contraction C = X^T Y.
//
// Some callers cannot allocate device memory while they call this library:
// code running inside a memory budget that another runtime owns (a framework
// allocator or pool that must see every allocation), code that must not
// trigger the implicit synchronisation of cudaMalloc/cudaFree, and code that
// cannot pass a workspace through its own fixed interface.  For them this
// file keeps the split-K partial sums of the contraction in a file-scope
// device array instead of a caller workspace or cudaMallocAsync.
//
// The array is fixed-size: every GPU that loads the library holds it until the
// process exits.  Host code only sees a host-side stand-in for its name, so
// the device address is looked up with cudaGetSymbolAddress once per device
// (with that device current) and that address is what the kernels receive.
#include <mutex>

#include "../../include/feast_gb300.h"
#include "feast_internal.cuh"

namespace feast {
const char* set_last_error(const char* msg);
}

namespace {

// 16 MiB of split-K partial sums (2 Mi doubles).
constexpr size_t kGramScratchDoubles = (size_t)2 * 1024 * 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_gram_scratch[kGramScratchDoubles];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_gram_scratch on the current device (looked up on the
// first call for each device).
cudaError_t scratch_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = (double*)p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int feast_gram_noalloc_dev(int n, int m, const double* X, const double* Y, double* C, void* stream)
{
    using namespace feast;
    cudaStream_t s = (cudaStream_t)stream;
    if (n <= 0) {
        set_last_error("feast_gram_noalloc_dev: n must be positive");
        return -101;
    }
    if (m <= 0 || (size_t)m * m > kGramScratchDoubles) {
        set_last_error("feast_gram_noalloc_dev: m exceeds the fixed scratch (m*m must be <= 2097152, m <= 1448)");
        return -102;
    }
    // as many row splits as the normal path uses, limited by the fixed array
    int ks = 1;
    gram_partial_doubles(n, m, &ks, num_sms());
    const size_t fit = kGramScratchDoubles / ((size_t)m * m);
    if ((size_t)ks > fit) ks = (int)fit;
    if (ks < 1) ks = 1;
    double* part = nullptr;
    cudaError_t e = scratch_address(&part);
    if (e == cudaSuccess) e = launch_gram_f64(n, m, X, Y, C, part, ks, 1, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return -4;
    }
    return 0;
}
