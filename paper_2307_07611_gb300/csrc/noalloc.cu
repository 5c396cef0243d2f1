// noalloc.cu -- tri_inv_noalloc: the plain triangular inverse for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: an application whose own memory manager has
// already reserved the device's memory (an allocation from inside the library would
// fail, or fragment that manager's pool), or latency-critical code that must neither
// block in the CUDA allocator nor handle an allocation failure in the middle of its
// work.  For them this entry point runs the same plain TRI_F32 / TRI_F64 inverse as
// tri_inv(), but the scratch of the level products lives in the fixed device array
// below instead of coming from the library's stream-ordered pool.  The caller still passes
// the matrix.
//
// The array (TRI_NOALLOC_SCRATCH_BYTES) exists on every GPU that loads the library and
// stays allocated until the process exits.  Host code cannot use the array's name as a
// device address (in host code it names a host-side stand-in), so the first call on each
// device looks the address up with cudaGetSymbolAddress, with that device current, and
// caches it for the life of the process (the cache does not survive cudaDeviceReset,
// after which the module is loaded again at another address).  Every call on a device
// shares the array and finds the previous call's contents in it; the inverse writes every
// scratch element before reading it within a call, so nothing needs clearing.  Calls
// whose GPU work can overlap race on the array.
#include <mutex>

#include "internal.cuh"

namespace triinv {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[TRI_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64];

// Device address of this device's scratch array (looked up once per device).
tri_status noalloc_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TRI_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TRI_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return TRI_OK;
}

}  // namespace
}  // namespace triinv

extern "C" tri_status tri_inv_noalloc(tri_uplo uplo, tri_diag diag, int64_t n, void *a,
                                      int64_t lda, tri_dtype dtype, void *stream) {
    using namespace triinv;
    if ((uplo != TRI_LOWER && uplo != TRI_UPPER) || (diag != TRI_NONUNIT && diag != TRI_UNIT) ||
        n < 0)
        return TRI_ERR_ARG;
    if (dtype == TRI_F32_MIXED) return TRI_ERR_UNSUPPORTED;
    if (dtype != TRI_F32 && dtype != TRI_F64) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    if (!a || lda < (n > 1 ? n : 1)) return TRI_ERR_ARG;
    const size_t need = tri_inv_workspace_size(n, dtype);
    if (need > (size_t)TRI_NOALLOC_SCRATCH_BYTES) return TRI_ERR_ARG;
    void *scratch = nullptr;
    tri_status st = noalloc_scratch(&scratch);
    if (st != TRI_OK) return st;
    return tri_inv_ex(uplo, diag, n, a, lda, dtype, scratch, (size_t)TRI_NOALLOC_SCRATCH_BYTES, nullptr,
                      stream);
}
