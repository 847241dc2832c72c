// lu_noalloc.cu -- dense LU factorisation entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc while they run: codes that reserve the device's
// memory up front for their own pool (a cudaMalloc would fail, or fragment the pool),
// and latency-critical loops that must not allocate after start-up (cudaMalloc and
// cudaFree can synchronise the device).  nebem_lu_factor_device_noalloc gives them the
// same factorisation as nebem_lu_factor_device with its work space (the inverse of the
// diagonal block, the row-panel staging buffer, the pivot-search partials and the
// singularity flag) in one file-scope device array instead of a per-call allocation.
//
// The array is a static __device__ object of this library: every GPU that loads the
// library holds it (about 2.1 MB) until the process exits, and all calls on a device
// share it, so calls whose GPU work overlaps in time race on it.  In host code its name
// is only a host-side stand-in: every call asks the runtime for the array's address in
// the context current on the calling thread (cudaGetSymbolAddress, which allocates
// nothing).  The address is not cached: a cached one would go stale after a
// cudaDeviceReset, and would belong to another context when the caller makes a
// non-primary context current (each context holds its own instance of the array).
#include "context.h"

namespace nb {

namespace {

constexpr int64_t kNoAllocMaxN = 4096;
constexpr int kNoAllocBlock = 64;
// lu_work_elems(kNoAllocMaxN, kNoAllocBlock) doubles of work space, then the flag
constexpr size_t kWorkDoubles = (size_t)4 * kNoAllocBlock * kNoAllocBlock + (size_t)kNoAllocBlock * kNoAllocMaxN + 16 +
                                (size_t)256 * 4 + 16 + (2 * 128 + 16);
constexpr size_t kScratchDoubles = kWorkDoubles + 32;  // + flags (two ints)

static __device__ __align__(256) double g_lu_scratch[kScratchDoubles];

// Device address of the array in the current context (looked up on every call).
int scratch_address(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_lu_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_lu_scratch)");
    *out = static_cast<double*>(p);
    return NEBEM_OK;
}

}  // namespace

}  // namespace nb

using namespace nb;

extern "C" int nebem_lu_factor_device_noalloc(double* d_A, int64_t n, int32_t* d_piv, void* stream) {
    if (!d_A || !d_piv || n <= 0) return fail(NEBEM_INVALID_ARG, "bad argument");
    if (n > kNoAllocMaxN)
        return fail(NEBEM_TOO_LARGE, "nebem_lu_factor_device_noalloc handles n <= 4096 (static work space)");
    static_assert(kWorkDoubles >= 4 * 64 * 64 + 64 * 4096 + 16 + 256 * 4 + 16 + 272, "work space too small");
    double* scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc) return rc;
    int* info = reinterpret_cast<int*>(scratch + kWorkDoubles);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = lu_factor_f64(d_A, n, d_piv, kNoAllocBlock, scratch, info, s);  // clears the flag first
    if (e != cudaSuccess) return cuda_fail(e, "lu_factor_f64");
    int h_info = 0;
    e = cudaMemcpyAsync(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "nebem_lu_factor_device_noalloc");
    if (h_info) return fail(NEBEM_SINGULAR, "zero pivot at column " + std::to_string(h_info - 1));
    return NEBEM_OK;
}
