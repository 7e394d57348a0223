// Shared device helpers of the CUDA library: complex arithmetic on
// float2/double2, the packed-panel layout of T, and error plumbing.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <type_traits>

namespace pseudo {

// Counts every kernel launch the library makes (process-wide).
void note_launch();
// kernels run by graph replays (counted on the device), and this thread's
// running count of note_launch calls (kernels per captured graph body)
void note_launches(long long k);
long long thread_launch_count();

// Raises a kernel's dynamic shared-memory limit before its first launch on
// each device (the attribute is per device; `done` holds one bit per device
// ordinal).  Host threads may race here: a thread sees a device's bit only
// after a completed set, and a repeated set is harmless.
template <typename Kernel>
inline void smem_attr_once(Kernel kernel, int bytes, std::atomic<uint64_t> &done) {
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done.fetch_or(bit, std::memory_order_release);
}

// ---------------------------------------------------------------- complex
template <typename real> struct cx;
template <> struct cx<double> { using t = double2; };
template <> struct cx<float> { using t = float2; };
template <typename real> using cx_t = typename cx<real>::t;

template <typename real> __host__ __device__ __forceinline__ cx_t<real> mk(real a, real b) {
    cx_t<real> r; r.x = a; r.y = b; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
    C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// acc += a * b
template <typename C> __host__ __device__ __forceinline__ void cfma(C &acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b
template <typename C> __host__ __device__ __forceinline__ void cfms(C &acc, C a, C b) {
    acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
template <typename C> __host__ __device__ __forceinline__ C cscale(C a, decltype(a.x) s) { a.x *= s; a.y *= s; return a; }
template <typename C> __host__ __device__ __forceinline__ decltype(C().x) cabs2(C a) { return a.x * a.x + a.y * a.y; }

// 1/d with scaling so that |d|^2 neither overflows nor underflows.
template <typename C> __device__ __forceinline__ C crecip(C d) {
    using real = decltype(d.x);
    real s = fmax(fabs(d.x), fabs(d.y));
    C r;
    if (s == real(0)) { r.x = real(0); r.y = real(0); return r; }
    real a = d.x / s, b = d.y / s;
    real den = (a * a + b * b) * s;
    r.x = a / den; r.y = -b / den;
    return r;
}

template <typename C> __device__ __forceinline__ C shfl_c(C v, int src) {
    v.x = __shfl_sync(0xffffffffu, v.x, src);
    v.y = __shfl_sync(0xffffffffu, v.y, src);
    return v;
}

// ------------------------------------------------------------ panel layout
// T is stored as row panels of PH = 64 rows.  Upper panels (for T - zI):
// panel P holds columns [64P, n_pad); lower panels (for (T - zI)^H, i.e. the
// rows of T^H) hold columns [0, 64P + 64).  Inside a panel, columns come in
// pairs: element (row i, column k) sits at pair*128 + 2*i + (k & 1), so one
// 16-byte (FP32) / 32-byte (FP64) load gives a lane the two columns of a pair
// and a warp's 32 lanes read consecutive memory.
constexpr int PH = 64;
__host__ __device__ __forceinline__ int64_t upper_panel_offset(int64_t P, int64_t n_pad) {
    return (int64_t)PH * (P * n_pad - (int64_t)PH * P * (P - 1) / 2);
}
__host__ __device__ __forceinline__ int64_t lower_panel_offset(int64_t P) {
    return (int64_t)PH * PH * P * (P + 1) / 2;
}
__host__ __device__ __forceinline__ int64_t packed_size(int64_t n_pad) {
    int64_t np = n_pad / PH;
    return upper_panel_offset(np, n_pad);  // same total for both layouts
}

}  // namespace pseudo
