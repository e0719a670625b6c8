// pscl_assign_sse_noalloc: nearest center and sum of squared errors of a set of points,
// for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code that runs under an allocator that
// owns the whole device (a framework's caching allocator, a fixed memory plan), real-time
// or embedded hosts that forbid allocation after start-up, or code paths where an
// allocation would synchronise the device.  This entry point runs the same kernel as the
// SSE step of pscl_cluster, but its scratch (one float64 partial sum per thread block and a
// completion ticket) lives in the file-scope array below instead of memory the library
// allocates.  The caller supplies the points, the centers and the two outputs.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "pscl_internal.cuh"

namespace pscl {
namespace {

constexpr int kNoAllocMaxBlocks = 4096;               // partial sums the scratch can hold
constexpr size_t kNoAllocBytes = kNoAllocMaxBlocks * sizeof(double) + 256;
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: [partials (kNoAllocMaxBlocks doubles) | ticket].
// In host code this name is only a stand-in for the device array; the device address is
// obtained with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_sse_scratch[kNoAllocBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

// The unique id of the calling thread's current context (cuCtxGetId; ids are never reused
// within a process), 0 if there is none or the driver cannot say.
unsigned long long current_ctx_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static const GetCurrent get_cur = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        cudaGetLastError();
        return reinterpret_cast<GetCurrent>(f);
    }();
    static const GetId get_id = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        cudaGetLastError();
        return reinterpret_cast<GetId>(f);
    }();
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// With the device current: the device address of the scratch array in the current
// context, looked up again whenever the context differs from the one it was found in
// (a device reset or a rebuilt primary context loads the module afresh, possibly at
// another address).
cudaError_t scratch_for_device(int dev, void **addr, int *sms)
{
    std::lock_guard<std::mutex> lock(g_setup_mu);
    const unsigned long long id = current_ctx_id();
    if (!g_scratch_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sse_scratch);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_sm_count[dev] = n;
        g_scratch_addr[dev] = p;
        g_ctx_id[dev] = current_ctx_id();      // the lookup made the context current if it was not
    }
    *addr = g_scratch_addr[dev];
    *sms = g_sm_count[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace pscl

using namespace pscl;

extern "C" int pscl_assign_sse_noalloc(const float *points, int64_t n, int32_t d, const float *centers,
                                       int32_t k, int32_t *labels, double *sse, void *stream)
{
    auto fail = [](int code, const char *msg) {
        set_last_error(msg);
        return code;
    };
    if (!points || !centers || !labels || !sse) return fail(PSCL_EINVAL, "pscl_assign_sse_noalloc: NULL pointer");
    if (n < 1 || n > (int64_t)INT32_MAX) return fail(PSCL_EINVAL, "pscl_assign_sse_noalloc: n outside 1..2^31-1");
    if (d < 1 || d > kMaxD) return fail(PSCL_EINVAL, "pscl_assign_sse_noalloc: d outside 1..1024");
    if (k < 1 || k > kMaxK) return fail(PSCL_EINVAL, "pscl_assign_sse_noalloc: k outside 1..4096");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(PSCL_ECUDA, "pscl_assign_sse_noalloc: no usable current device");
    }
    void *scratch = nullptr;
    int sms = 0;
    if (scratch_for_device(dev, &scratch, &sms) != cudaSuccess) {
        cudaGetLastError();
        return fail(PSCL_ECUDA, "pscl_assign_sse_noalloc: cudaGetSymbolAddress of the scratch array failed");
    }
    if (sse_grid(n, sms) > kNoAllocMaxBlocks)
        return fail(PSCL_EINVAL, "pscl_assign_sse_noalloc: the launch needs more partial sums than the scratch holds");
    double *partials = static_cast<double *>(scratch);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(scratch) +
                                                    kNoAllocMaxBlocks * sizeof(double));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the ticket counts finished blocks and must start at zero (the partials are overwritten)
    if (cudaMemsetAsync(ticket, 0, sizeof(uint32_t), st) != cudaSuccess) {
        cudaGetLastError();
        return fail(PSCL_ECUDA, "pscl_assign_sse_noalloc: clearing the scratch failed");
    }
    KTimer kt;
    cudaError_t e = launch_final_sse(points, n, d, centers, k, labels, partials, sse, ticket, sms, st, &kt);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PSCL_ECUDA, cudaGetErrorString(e));
    }
    return PSCL_OK;
}
