// pseudo_solve_noalloc: the FP64 multi-shift triangular solve for callers
// that cannot allocate device memory.  The paper has no counterpart; this is a
// library-usage entry point.
//
// The solve needs scratch memory (a compact copy of the solved columns, one
// n_pad x 8 block per group of 8 columns, n_pad = n rounded up to 128).
// pseudo_solve takes it from a caller-provided workspace; this entry point
// uses a fixed array in the library's own device memory instead, so a caller
// with no allocator at all (a process that reserved its whole device-memory
// budget up front, or a latency-critical loop that must not call
// cudaMalloc/cudaFree because they can synchronise the device) can still run
// solves.
#include <mutex>

#include "common.cuh"
#include "driver.h"
#include "internal.h"

namespace pseudo {

// 2^20 complex doubles = 16 MiB.  Every GPU that loads the library holds this
// array until the process exits.
constexpr size_t NOALLOC_SCRATCH_ELEMS = (size_t)1 << 20;
static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_SCRATCH_ELEMS];

// In host code g_noalloc_scratch names a host-side stand-in, not the device
// array, so its device address is looked up once per device (with that
// device current) and cached here.  The cache does not survive a device
// reset (cudaDeviceReset or a teardown of the primary context unloads the
// module): the header tells callers not to use this entry point after one.
constexpr int NOALLOC_MAX_DEVICES = 64;
static double2 *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
static std::mutex g_noalloc_mu;

static int noalloc_scratch(int dev, double2 **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return set_err(PSEUDO_ERR_UNSUPPORTED, "device id %d out of range", dev);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_ptr[dev] = (double2 *)p;
    }
    *out = g_noalloc_ptr[dev];
    return PSEUDO_OK;
}

}  // namespace pseudo

using namespace pseudo;

extern "C" int pseudo_solve_noalloc(pseudo_handle h, pseudo_c64 *X, const pseudo_c64 *z, int64_t ncols, int adjoint,
                                    void *stream) {
    clear_err();
    if (misaligned(X, 16) || misaligned(z, 16))
        return set_err(PSEUDO_ERR_ARG, "X and z must be 16-byte aligned (complex doubles)");
    if (!h || !X || !z || ncols < 0) return set_err(PSEUDO_ERR_ARG, "bad argument");
    if (h->rect) return set_err(PSEUDO_ERR_UNSUPPORTED, "shifted solves need a square handle (m = n)");
    if (ncols == 0) return PSEUDO_OK;
    // Each group of 8 columns needs at least 128 scratch elements, so more
    // than NOALLOC_SCRATCH_ELEMS columns can never fit; rejecting them here
    // also keeps the size product below from overflowing.
    if ((uint64_t)ncols > NOALLOC_SCRATCH_ELEMS)
        return set_err(PSEUDO_ERR_ARG, "pseudo_solve_noalloc: %lld columns exceed the fixed scratch of %zu elements",
                       (long long)ncols, NOALLOC_SCRATCH_ELEMS);
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
    if (cur != h->dev) return set_err(PSEUDO_ERR_ARG, "the handle's device (%d) must be current (is %d)", h->dev, cur);
    const size_t need = trsv_scratch_bytes(0, h->n_pad, ncols) / sizeof(double2);
    if (need > NOALLOC_SCRATCH_ELEMS)
        return set_err(PSEUDO_ERR_ARG,
                       "pseudo_solve_noalloc: %lld columns of order %d need %zu scratch elements, more than the fixed "
                       "%zu (use pseudo_solve with a workspace)",
                       (long long)ncols, h->n, need, NOALLOC_SCRATCH_ELEMS);
    double2 *xs = nullptr;
    const int rc = noalloc_scratch(cur, &xs);
    if (rc != PSEUDO_OK) return rc;
    // Every scratch row is written by the solve before it is read, so the
    // contents left by an earlier call need no clearing.
    const int lower = adjoint ? 1 : 0;
    e = launch_trsv64(lower ? h->L64 : h->U64, h->n, h->n_pad, lower, nullptr, (const double2 *)z, (int)ncols, nullptr,
                      (double2 *)X, ncols, xs, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_err(e, "pseudo_solve_noalloc");
    h->stats.sv_R += ncols;
    return PSEUDO_OK;
}
