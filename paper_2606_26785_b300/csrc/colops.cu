// Column-wise vector kernels on row-major n x S blocks (one column per grid
// point): norms, FP64 <-> FP32 conversion with per-column scaling (the
// correction solves of iterative refinement), accumulation, Rayleigh quotient
// and residual of the returned singular vector, and the final scatter of
// sigma / residual / flags / epsilon-membership into the caller's arrays.
// CTAs cover 32 consecutive columns (lane = column), warps split the rows.
#include "common.cuh"
#include "internal.h"

namespace pseudo {

constexpr int CW = 8;  // warps per CTA

__device__ __forceinline__ double block_col_sum(double v, double (*sh)[32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    sh[warp][lane] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < CW; ++w) t += sh[w][lane];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(CW * 32)
colnorm2_kernel(const double2 *__restrict__ X, int n, int S, const int *__restrict__ mask, double *__restrict__ out) {
    __shared__ double sh[CW][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const bool on = c < S && (!mask || mask[c]);
    double s = 0.0;
    if (on)
        for (int i = warp; i < n; i += CW) { const double2 v = X[(int64_t)i * S + c]; s += v.x * v.x + v.y * v.y; }
    s = block_col_sum(s, sh);
    if (on && warp == 0) out[c] = s;
}

// D = R / sqrt(rn2)  (FP32), 0 where rn2 == 0
__global__ void __launch_bounds__(CW * 32)
scale_to32_kernel(const double2 *__restrict__ R, int n, int S, const int *__restrict__ mask,
                  const double *__restrict__ rn2, float2 *__restrict__ D) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    if (c >= S || (mask && !mask[c])) return;
    const double inv = rn2[c] > 0.0 ? 1.0 / sqrt(rn2[c]) : 0.0;
    for (int i = warp; i < n; i += CW) {
        const double2 v = R[(int64_t)i * S + c];
        D[(int64_t)i * S + c] = make_float2((float)(v.x * inv), (float)(v.y * inv));
    }
}

// X += sqrt(rn2) * D
__global__ void __launch_bounds__(CW * 32)
acc_from32_kernel(double2 *__restrict__ X, int n, int S, const int *__restrict__ mask, const double *__restrict__ rn2,
                  const float2 *__restrict__ D) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    if (c >= S || (mask && !mask[c])) return;
    const double sc = sqrt(rn2[c]);
    for (int i = warp; i < n; i += CW) {
        const float2 d = D[(int64_t)i * S + c];
        double2 x = X[(int64_t)i * S + c];
        x.x += sc * (double)d.x; x.y += sc * (double)d.y;
        X[(int64_t)i * S + c] = x;
    }
}

// X /= ||X|| per column
__global__ void __launch_bounds__(CW * 32)
normalize_kernel(double2 *__restrict__ X, int n, int S, const int *__restrict__ mask) {
    __shared__ double sh[CW][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const bool on = c < S && (!mask || mask[c]);
    double s = 0.0;
    if (on)
        for (int i = warp; i < n; i += CW) { const double2 v = X[(int64_t)i * S + c]; s += v.x * v.x + v.y * v.y; }
    s = block_col_sum(s, sh);
    if (!on) return;
    const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    for (int i = warp; i < n; i += CW) { double2 v = X[(int64_t)i * S + c]; v.x *= inv; v.y *= inv; X[(int64_t)i * S + c] = v; }
}

// For unit x = U[:, c], Y = (T - zI) x and NX = (T - zI)^H Y:
//   s2 = ||Y||^2 (Rayleigh quotient of N(z) at x), r = ||NX - s2 x||.
__global__ void __launch_bounds__(CW * 32)
rq_residual_kernel(const double2 *__restrict__ U, const double2 *__restrict__ Y, const double2 *__restrict__ NX, int n,
                   int ny, int S, const int *__restrict__ mask, double *__restrict__ s2_out, double *__restrict__ r_out) {
    __shared__ double sh[CW][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const bool on = c < S && (!mask || mask[c]);
    double s = 0.0;
    if (on)
        for (int i = warp; i < ny; i += CW) { const double2 v = Y[(int64_t)i * S + c]; s += v.x * v.x + v.y * v.y; }
    const double s2 = block_col_sum(s, sh);
    double r = 0.0;
    if (on)
        for (int i = warp; i < n; i += CW) {
            const double2 a = NX[(int64_t)i * S + c], u = U[(int64_t)i * S + c];
            const double dx = a.x - s2 * u.x, dy = a.y - s2 * u.y;
            r += dx * dx + dy * dy;
        }
    r = block_col_sum(r, sh);
    if (on && warp == 0) { s2_out[c] = s2; r_out[c] = sqrt(r); }
}

// Scatter results of a wave of S points starting at point w0.
//   sig_src: 0 -> sigma = 1/sqrt(theta); 1 -> sigma = sqrt(s2)
__global__ void finalize_kernel(int S, int64_t w0, const double2 *__restrict__ z, const double *__restrict__ theta,
                                const double *__restrict__ s2, const double *__restrict__ rr, const int *__restrict__ active,
                                const int *__restrict__ extra_flags, int sig_src, double norm2,
                                const double *__restrict__ eps, int neps, double *__restrict__ sigma_out,
                                double *__restrict__ res_out, int32_t *__restrict__ flags_out,
                                uint32_t *__restrict__ member_out, int base_flags, int *__restrict__ nbad) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= S) return;
    double sig = sig_src == 0 ? (theta[c] > 0.0 ? 1.0 / sqrt(theta[c]) : 0.0) : sqrt(fmax(s2[c], 0.0));
    const double2 zz = z[c];
    const double mz = norm2 + sqrt(zz.x * zz.x + zz.y * zz.y);
    const double sref = sig_src == 0 ? sqrt(fmax(s2[c], 0.0)) : sig;
    int fl = base_flags | (extra_flags ? extra_flags[c] : 0);
    if (active && active[c] == -1) { fl |= PSEUDO_PT_NOT_CONVERGED; atomicAdd(nbad, 1); }
    sigma_out[w0 + c] = sig;
    if (res_out) res_out[w0 + c] = sref > 0.0 ? rr[c] / (sref * mz) : 0.0;
    if (flags_out) flags_out[w0 + c] = fl;
    if (member_out) {
        uint32_t m = 0;
        for (int e = 0; e < neps; ++e) m |= (sig < eps[e] ? 1u : 0u) << e;
        member_out[w0 + c] = m;
    }
}

__global__ void fill_int_kernel(int *a, int n, int v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

__global__ void nonfinite_kernel(const double2 *__restrict__ a, int64_t cnt, int *bad) {
    int loc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(a[i].x) || !isfinite(a[i].y)) loc = 1;
    if (__syncthreads_or(loc) && threadIdx.x == 0) atomicOr(bad, 1);
}

// ------------------------------------------------------------ launchers
static inline unsigned cgroups(int S) { return (unsigned)((S + 31) / 32); }
void launch_colnorm2(const double2 *X, int n, int S, const int *mask, double *out, cudaStream_t s) {
    note_launch(); colnorm2_kernel<<<cgroups(S), CW * 32, 0, s>>>(X, n, S, mask, out);
}
void launch_scale_to32(const double2 *R, int n, int S, const int *mask, const double *rn2, float2 *D, cudaStream_t s) {
    note_launch(); scale_to32_kernel<<<cgroups(S), CW * 32, 0, s>>>(R, n, S, mask, rn2, D);
}
void launch_acc_from32(double2 *X, int n, int S, const int *mask, const double *rn2, const float2 *D, cudaStream_t s) {
    note_launch(); acc_from32_kernel<<<cgroups(S), CW * 32, 0, s>>>(X, n, S, mask, rn2, D);
}
void launch_normalize(double2 *X, int n, int S, const int *mask, cudaStream_t s) {
    note_launch(); normalize_kernel<<<cgroups(S), CW * 32, 0, s>>>(X, n, S, mask);
}
void launch_rq_residual(const double2 *U, const double2 *Y, const double2 *NX, int n, int S, const int *mask,
                        double *s2, double *r, cudaStream_t s, int ny) {
    note_launch(); rq_residual_kernel<<<cgroups(S), CW * 32, 0, s>>>(U, Y, NX, n, ny > 0 ? ny : n, S, mask, s2, r);
}
void launch_finalize(int S, int64_t w0, const double2 *z, const double *theta, const double *s2, const double *rr,
                     const int *active, const int *extra_flags, int sig_src, double norm2, const double *eps, int neps,
                     double *sigma_out, double *res_out, int32_t *flags_out, uint32_t *member_out, int base_flags,
                     int *nbad, cudaStream_t s) {
    note_launch(); finalize_kernel<<<(S + 127) / 128, 128, 0, s>>>(S, w0, z, theta, s2, rr, active, extra_flags, sig_src, norm2, eps,
                                                    neps, sigma_out, res_out, flags_out, member_out, base_flags, nbad);
}
void launch_fill_int(int *a, int n, int v, cudaStream_t s) {
    if (n > 0) { note_launch(); fill_int_kernel<<<(n + 255) / 256, 256, 0, s>>>(a, n, v); }
}
void launch_nonfinite(const double2 *a, int64_t cnt, int *bad, cudaStream_t s) {
    note_launch(); nonfinite_kernel<<<296, 256, 0, s>>>(a, cnt, bad);
}

}  // namespace pseudo

namespace pseudo {
__global__ void cvt64to32_kernel(const double2 *__restrict__ a, float2 *__restrict__ b, int64_t cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void cvt32to64_kernel(const float2 *__restrict__ a, double2 *__restrict__ b, int64_t cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = make_double2((double)a[i].x, (double)a[i].y);
}
void launch_convert_64_to_32(const double2 *a, float2 *b, int64_t cnt, cudaStream_t s) {
    if (cnt > 0) { note_launch(); cvt64to32_kernel<<<1184, 256, 0, s>>>(a, b, cnt); }
}
void launch_convert_32_to_64(const float2 *a, double2 *b, int64_t cnt, cudaStream_t s) {
    if (cnt > 0) { note_launch(); cvt32to64_kernel<<<1184, 256, 0, s>>>(a, b, cnt); }
}
}  // namespace pseudo
