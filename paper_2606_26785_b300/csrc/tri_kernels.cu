// Multi-shift triangular kernels on the packed panels of T.
//
//  * pack_panels       : T (column-major FP64) -> upper panels of T and lower
//                        panels of T^H, in FP64 and FP32.
//  * trsv_ms           : (T - z_c I) x_c = b_c  or  (T - z_c I)^H x_c = b_c for
//                        many columns c at once, each with its own shift: the
//                        R(z)^{-1} / R(z)^{-*} applications of Alg. 3 and of the
//                        inverse-Lanczos comparator (sv_R in Table 2).
//  * trmv_ms (FP64)    : y_c = b_c - (T - z_c I)^{op} x_c  (or without b): the
//                        refinement residual and the products T V, T^H V of
//                        Alg. 2 (mv_M in Table 2).
//
// Blocking: a CTA owns R right-hand sides.  Row panels of 64 rows are solved
// one after another (bottom-up for T, top-down for T^H).  For a panel, the
// off-diagonal contribution sum_K T_IK x_K is split over the CTA's warps (lane
// l of a warp holds rows l and l+32 of the panel, R accumulators each), summed
// through shared memory, and warp 0 then solves the 64 x 64 diagonal block
// with warp shuffles.  Solutions already computed are read from a compact
// per-CTA copy (scratch: 64-row-padded n x R per CTA), so every x_k load is a
// contiguous broadcast of R values.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace pseudo {

template <typename real> __device__ __forceinline__ cx_t<real> cvt(double2 v);
template <> __device__ __forceinline__ double2 cvt<double>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt<float>(double2 v) { return make_float2((float)v.x, (float)v.y); }

template <typename real>
__global__ void pack_panels_kernel(const double2 *__restrict__ T, int64_t ldT, int n, int n_pad,
                                   cx_t<real> *__restrict__ U, cx_t<real> *__restrict__ L) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_pad * n_pad) return;
    const int k = (int)(idx / n_pad), i = (int)(idx % n_pad);
    const int P = i / PH, li = i % PH;
    if (k >= P * PH) {  // row i of T, column k (upper triangle only)
        double2 v = (i < n && k < n && i <= k) ? T[(int64_t)k * ldT + i] : make_double2(0.0, 0.0);
        int64_t rel = k - (int64_t)P * PH;
        U[upper_panel_offset(P, n_pad) + (rel >> 1) * (2 * PH) + 2 * li + (rel & 1)] = cvt<real>(v);
    }
    if (k < (P + 1) * PH) {  // row i of T^H, column k: conj(T(k, i)) for k <= i
        double2 v = (i < n && k < n && k <= i) ? T[(int64_t)i * ldT + k] : make_double2(0.0, 0.0);
        v.y = -v.y;
        L[lower_panel_offset(P) + (int64_t)(k >> 1) * (2 * PH) + 2 * li + (k & 1)] = cvt<real>(v);
    }
}

void launch_pack_panels(const double2 *T, int64_t ldT, int n, int n_pad, double2 *U64, double2 *L64,
                        float2 *U32, float2 *L32, cudaStream_t s) {
    int64_t tot = (int64_t)n_pad * n_pad;
    int th = 256;
    int64_t bl = (tot + th - 1) / th;
    note_launch(); pack_panels_kernel<double><<<(unsigned)bl, th, 0, s>>>(T, ldT, n, n_pad, U64, L64);
    note_launch(); pack_panels_kernel<float><<<(unsigned)bl, th, 0, s>>>(T, ldT, n, n_pad, U32, L32);
}

// ------------------------------------------------------------------ solve
template <typename real, int R, int NW>
__global__ void __launch_bounds__(NW * 32)
trsv_ms_kernel(const cx_t<real> *__restrict__ Pn, int n, int n_pad, int lower,
               const int *__restrict__ cols, const double2 *__restrict__ zc, int ncols_host,
               const int *__restrict__ ncols_dev, cx_t<real> *X, int64_t ldx, cx_t<real> *xs_all, int cmin,
               int cmax) {
    using C = cx_t<real>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *red = reinterpret_cast<C *>(smem_raw);   // [NW][PH][R]
    C *s_dinv = red + NW * PH * R;               // [PH][R]
    __shared__ int s_col[R];
    __shared__ double2 s_z[R];

    const int ncols = ncols_dev ? *ncols_dev : ncols_host;
    const int g = blockIdx.x;
    // [cmin, cmax]: the live counts this column-group width serves (one of
    // several launches over an upper bound of the count; the others leave)
    if (g * R >= ncols || ncols < cmin || ncols > cmax) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < R) {
        int pos = g * R + threadIdx.x;
        int c = -1;
        double2 z = make_double2(0.0, 0.0);
        if (pos < ncols) { c = cols ? cols[pos] : pos; z = zc[c]; }
        if (lower) z.y = -z.y;  // (T - zI)^H = T^H - conj(z) I
        s_col[threadIdx.x] = c;
        s_z[threadIdx.x] = z;
    }
    __syncthreads();
    C *xs = xs_all + (int64_t)g * n_pad * R;
    const int npan = n_pad / PH;

    for (int step = 0; step < npan; ++step) {
        const int P = lower ? step : npan - 1 - step;
        const C *pan = Pn + (lower ? lower_panel_offset(P) : upper_panel_offset(P, n_pad));
        int kp0, kp1, kcol0;
        if (!lower) { kp0 = PH / 2; kp1 = (n_pad - P * PH) / 2; kcol0 = P * PH; }
        else { kp0 = 0; kp1 = P * PH / 2; kcol0 = 0; }

        C acc[2][R];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int c = 0; c < R; ++c) acc[q][c] = mk<real>(0, 0);

        const int nk = kp1 - kp0;
        const int per = (nk + NW - 1) / NW;
        const int a = kp0 + warp * per;
        const int b = min(kp1, a + per);
#pragma unroll 2
        for (int kp = a; kp < b; ++kp) {
            const C *tp = pan + (int64_t)kp * (2 * PH) + 2 * lane;
            const C t00 = tp[0], t01 = tp[1], t10 = tp[64], t11 = tp[65];
            const C *x0 = xs + (int64_t)(kcol0 + 2 * kp) * R;
#pragma unroll
            for (int c = 0; c < R; ++c) {
                const C xa = x0[c], xb = x0[R + c];
                cfma(acc[0][c], t00, xa); cfma(acc[0][c], t01, xb);
                cfma(acc[1][c], t10, xa); cfma(acc[1][c], t11, xb);
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int c = 0; c < R; ++c) red[((warp * PH) + lane + 32 * q) * R + c] = acc[q][c];
        // inverse diagonal of this panel for every column
        for (int e = threadIdx.x; e < PH * R; e += NW * 32) {
            const int li = e / R, c = e % R, row = P * PH + li;
            C d = mk<real>(0, 0);
            if (row < n) {
                const int64_t dp = lower ? (int64_t)(P * 32 + (li >> 1)) : (int64_t)(li >> 1);
                const C t = pan[dp * (2 * PH) + 2 * li + (li & 1)];
                // 1/(t_ii - z) in the kernel's own precision (a scaled complex
                // reciprocal: no FP64 instruction in the FP32 solve)
                d = crecip(mk<real>(t.x - (real)s_z[c].x, t.y - (real)s_z[c].y));
            }
            s_dinv[li * R + c] = d;
        }
        __syncthreads();

        // diagonal block: warp w solves columns [w*CPW, w*CPW + CPW) of the
        // CTA's R right-hand sides (every warp busy when R >= NW)
        constexpr int CPW = (R + NW - 1) / NW;
        const int c0 = warp * CPW;
        if (c0 < R) {
            C tot[2][CPW];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int row = P * PH + lane + 32 * q;
#pragma unroll
                for (int cc = 0; cc < CPW; ++cc) {
                    const int c = c0 + cc;
                    C bv = mk<real>(0, 0);
                    if (c < R) {
                        if (row < n && s_col[c] >= 0) bv = X[(int64_t)row * ldx + s_col[c]];
#pragma unroll
                        for (int w = 0; w < NW; ++w) bv = csub(bv, red[((w * PH) + lane + 32 * q) * R + c]);
                    }
                    tot[q][cc] = bv;
                }
            }
            if (!lower) {
#pragma unroll
                for (int q = 1; q >= 0; --q) {
                    for (int l = 31; l >= 0; --l) {
                        const int i = 32 * q + l;
                        const C *dcol = pan + (int64_t)(i >> 1) * (2 * PH) + (i & 1);
                        const C t0 = dcol[2 * lane], t1 = dcol[2 * (lane + 32)];
#pragma unroll
                        for (int cc = 0; cc < CPW; ++cc) {
                            const int c = min(c0 + cc, R - 1);
                            C xi = shfl_c(cmul(tot[q][cc], s_dinv[i * R + c]), l);
                            if (lane == l) tot[q][cc] = xi;
                            if (q == 1) {
                                cfms(tot[0][cc], t0, xi);
                                if (lane < l) cfms(tot[1][cc], t1, xi);
                            } else {
                                if (lane < l) cfms(tot[0][cc], t0, xi);
                            }
                        }
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    for (int l = 0; l < 32; ++l) {
                        const int i = 32 * q + l;
                        const C *dcol = pan + (int64_t)(P * 32 + (i >> 1)) * (2 * PH) + (i & 1);
                        const C t0 = dcol[2 * lane], t1 = dcol[2 * (lane + 32)];
#pragma unroll
                        for (int cc = 0; cc < CPW; ++cc) {
                            const int c = min(c0 + cc, R - 1);
                            C xi = shfl_c(cmul(tot[q][cc], s_dinv[i * R + c]), l);
                            if (lane == l) tot[q][cc] = xi;
                            if (q == 0) {
                                if (lane > l) cfms(tot[0][cc], t0, xi);
                                cfms(tot[1][cc], t1, xi);
                            } else {
                                if (lane > l) cfms(tot[1][cc], t1, xi);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int row = P * PH + lane + 32 * q;
#pragma unroll
                for (int cc = 0; cc < CPW; ++cc) {
                    const int c = c0 + cc;
                    if (c >= R) continue;
                    const C v = row < n ? tot[q][cc] : mk<real>(0, 0);
                    xs[(int64_t)row * R + c] = v;
                    if (row < n && s_col[c] >= 0) X[(int64_t)row * ldx + s_col[c]] = v;
                }
            }
        }
        __syncthreads();
    }
}

template <typename real, int R, int NW>
static size_t trsv_smem() { return sizeof(cx_t<real>) * (size_t)(NW * PH * R + PH * R); }

template <typename real, int R, int NW>
static cudaError_t trsv_launch(const cx_t<real> *Pn, int n, int n_pad, int lower, const int *cols,
                               const double2 *zc, int ncols, const int *ncols_dev, cx_t<real> *X,
                               int64_t ldx, cx_t<real> *xs, cudaStream_t s, int cmin = 0,
                               int cmax = 0x7fffffff) {
    size_t sm = trsv_smem<real, R, NW>();
    static std::atomic<uint64_t> attr{0};
    smem_attr_once(trsv_ms_kernel<real, R, NW>, (int)sm, attr);
    int grid = (ncols + R - 1) / R;
    if (grid == 0) return cudaSuccess;
    note_launch(); trsv_ms_kernel<real, R, NW><<<grid, NW * 32, sm, s>>>(Pn, n, n_pad, lower, cols, zc, ncols, ncols_dev, X, ldx, xs,
                                                                  cmin, cmax);
    return cudaGetLastError();
}

// Column-group width of the solves: FP64 8 columns, FP32 16 columns per CTA.
constexpr int R64 = 8, R32 = 16, NW_SOLVE = 8;
int trsv_group_width(int fp32) { return fp32 ? R32 : R64; }

size_t trsv_scratch_bytes(int fp32, int64_t n_pad, int64_t ncols) {
    if (fp32) return trsv32_scratch_bytes(n_pad, ncols);  // shared with the tensor-core solve
    int64_t groups = (ncols + R64 - 1) / R64;
    return (size_t)groups * n_pad * R64 * sizeof(double2);
}

cudaError_t launch_trsv64(const double2 *Pn, int n, int n_pad, int lower, const int *cols, const double2 *zc,
                          int ncols, const int *ncols_dev, double2 *X, int64_t ldx, double2 *xs, cudaStream_t s) {
    // FP64 runs at 1/62 of FP32 here, so a few columns must still spread over
    // many SMs: narrower column groups when the launch is small (the scratch
    // of 8-column groups covers them)
    if (ncols <= 296)
        return trsv_launch<double, 1, NW_SOLVE>(Pn, n, n_pad, lower, cols, zc, ncols, ncols_dev, X, ldx, xs, s);
    if (ncols <= 1184)
        return trsv_launch<double, 2, NW_SOLVE>(Pn, n, n_pad, lower, cols, zc, ncols, ncols_dev, X, ldx, xs, s);
    return trsv_launch<double, R64, NW_SOLVE>(Pn, n, n_pad, lower, cols, zc, ncols, ncols_dev, X, ldx, xs, s);
}
cudaError_t launch_trsv64_bounded(const double2 *Pn, int n, int n_pad, int lower, const int *cols, const double2 *zc,
                                  int bound, const int *ncols_dev, double2 *X, int64_t ldx, double2 *xs,
                                  cudaStream_t s) {
    // the live count is known only on the device: one launch per column-group
    // width that a count up to `bound` may need, each serving its own range
    cudaError_t e = trsv_launch<double, 1, NW_SOLVE>(Pn, n, n_pad, lower, cols, zc, std::min(bound, 296), ncols_dev, X,
                                                     ldx, xs, s, 0, 296);
    if (e == cudaSuccess && bound > 296)
        e = trsv_launch<double, 2, NW_SOLVE>(Pn, n, n_pad, lower, cols, zc, std::min(bound, 1184), ncols_dev, X, ldx,
                                             xs, s, 297, 1184);
    if (e == cudaSuccess && bound > 1184)
        e = trsv_launch<double, R64, NW_SOLVE>(Pn, n, n_pad, lower, cols, zc, bound, ncols_dev, X, ldx, xs, s, 1185);
    return e;
}
cudaError_t launch_trsv32(const float2 *Pn, int n, int n_pad, int lower, const int *cols, const double2 *zc,
                          int ncols, const int *ncols_dev, float2 *X, int64_t ldx, float2 *xs, cudaStream_t s) {
    return trsv_launch<float, R32, NW_SOLVE>(Pn, n, n_pad, lower, cols, zc, ncols, ncols_dev, X, ldx, xs, s);
}

// ----------------------------------------------------------------- matvec
template <int R, int NW>
__global__ void __launch_bounds__(NW * 32)
trmv_ms_kernel(const double2 *__restrict__ Pn, int n, int n_pad, int lower, const int *__restrict__ cols,
               const double2 *__restrict__ zc, int ncols_host, const int *__restrict__ ncols_dev,
               const double2 *__restrict__ X, int64_t ldx, const double2 *__restrict__ B, int64_t ldb,
               double2 *__restrict__ Y, int64_t ldy, int subtract) {
    using C = double2;
    __shared__ C red[NW][PH][R];
    __shared__ int s_col[R];
    __shared__ double2 s_z[R];
    const int ncols = ncols_dev ? *ncols_dev : ncols_host;
    const int P = blockIdx.x, g = blockIdx.y;
    if (g * R >= ncols) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < R) {
        int pos = g * R + threadIdx.x;
        int c = -1;
        double2 z = make_double2(0.0, 0.0);
        if (pos < ncols) { c = cols ? cols[pos] : pos; if (zc) z = zc[c]; }
        if (lower) z.y = -z.y;
        s_col[threadIdx.x] = c;
        s_z[threadIdx.x] = z;
    }
    __syncthreads();
    const C *pan = Pn + (lower ? lower_panel_offset(P) : upper_panel_offset(P, n_pad));
    const int kp1 = lower ? (P + 1) * PH / 2 : (n_pad - P * PH) / 2;
    const int kcol0 = lower ? 0 : P * PH;
    C acc[2][R];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < R; ++c) acc[q][c] = make_double2(0.0, 0.0);
    const int per = (kp1 + NW - 1) / NW;
    const int a = warp * per, b = min(kp1, a + per);
    for (int kp = a; kp < b; ++kp) {
        const C *tp = pan + (int64_t)kp * (2 * PH) + 2 * lane;
        const C t00 = tp[0], t01 = tp[1], t10 = tp[64], t11 = tp[65];
        const int k0 = kcol0 + 2 * kp;
#pragma unroll
        for (int c = 0; c < R; ++c) {
            const int cc = s_col[c];
            C xa = make_double2(0.0, 0.0), xb = xa;
            if (cc >= 0) {
                if (k0 < n) xa = X[(int64_t)k0 * ldx + cc];
                if (k0 + 1 < n) xb = X[(int64_t)(k0 + 1) * ldx + cc];
            }
            cfma(acc[0][c], t00, xa); cfma(acc[0][c], t01, xb);
            cfma(acc[1][c], t10, xa); cfma(acc[1][c], t11, xb);
        }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < R; ++c) red[warp][lane + 32 * q][c] = acc[q][c];
    __syncthreads();
    for (int e = threadIdx.x; e < PH * R; e += NW * 32) {
        const int li = e / R, c = e % R, row = P * PH + li, cc = s_col[c];
        if (row >= n || cc < 0) continue;
        C y = make_double2(0.0, 0.0);
        for (int w = 0; w < NW; ++w) y = cadd(y, red[w][li][c]);
        const C xr = X[(int64_t)row * ldx + cc];
        cfms(y, s_z[c], xr);  // - z x_row
        if (subtract) y = csub(B[(int64_t)row * ldb + cc], y);
        Y[(int64_t)row * ldy + cc] = y;
    }
}

constexpr int RMV = 4, NW_MV = 4;
cudaError_t launch_trmv64(const double2 *Pn, int n, int n_pad, int lower, const int *cols, const double2 *zc,
                          int ncols, const int *ncols_dev, const double2 *X, int64_t ldx, const double2 *B,
                          int64_t ldb, double2 *Y, int64_t ldy, int subtract, cudaStream_t s) {
    if (ncols <= 0) return cudaSuccess;
    dim3 grid(n_pad / PH, (ncols + RMV - 1) / RMV);
    note_launch(); trmv_ms_kernel<RMV, NW_MV><<<grid, NW_MV * 32, 0, s>>>(Pn, n, n_pad, lower, cols, zc, ncols, ncols_dev, X, ldx,
                                                           B, ldb, Y, ldy, subtract);
    return cudaGetLastError();
}

// ------------------------------------------------- double-single product
// y_c = b_c - (T - z_c I)^{op} x_c (or without b) with T held as two FP32
// planes (T = T_hi + T_lo to 48 bits) and every product and sum carried in
// double-single arithmetic (Dekker's exact product through FMA and Knuth's
// two-sum), so that the FP32 pipes, 62x faster than FP64 on this GPU, give
// a result with relative error about 2^-46 instead of FP32's 2^-24.
struct dsf {
    float hi, lo;
};
__device__ __forceinline__ void ds_acc(dsf &s, float a_hi, float a_lo, float b_hi, float b_lo) {
    // s += a * b with a = a_hi + a_lo, b = b_hi + b_lo (a_lo * b_lo dropped)
    const float p = a_hi * b_hi;
    float e = fmaf(a_hi, b_hi, -p);
    e = fmaf(a_hi, b_lo, e);
    e = fmaf(a_lo, b_hi, e);
    const float t = s.hi + p;
    const float bp = t - s.hi;
    const float err = (s.hi - (t - bp)) + (p - bp);
    s.hi = t;
    s.lo += err + e;
}
__device__ __forceinline__ double ds_val(dsf s) { return (double)s.hi + (double)s.lo; }
__device__ __forceinline__ void ds_norm(dsf &s) {
    const float t = s.hi + s.lo;
    s.lo = s.lo - (t - s.hi);
    s.hi = t;
}

template <int R, int NW>
__global__ void __launch_bounds__(NW * 32)
trmv_ds_kernel(const float2 *__restrict__ Ph, const float2 *__restrict__ Pl, int n, int n_pad, int lower,
               const int *__restrict__ cols, const double2 *__restrict__ zc, int ncols,
               const double2 *__restrict__ X, const float2 *__restrict__ Xh, const float2 *__restrict__ Xl,
               int64_t ldx, const double2 *__restrict__ B, int64_t ldb, double2 *__restrict__ Y, int64_t ldy,
               int subtract) {
    __shared__ double2 red[NW][PH][R];
    __shared__ int s_col[R];
    __shared__ double2 s_z[R];
    const int P = blockIdx.x, g = blockIdx.y;
    if (g * R >= ncols) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < R) {
        int pos = g * R + threadIdx.x;
        int c = -1;
        double2 z = make_double2(0.0, 0.0);
        if (pos < ncols) { c = cols ? cols[pos] : pos; if (zc) z = zc[c]; }
        if (lower) z.y = -z.y;
        s_col[threadIdx.x] = c;
        s_z[threadIdx.x] = z;
    }
    __syncthreads();
    const int64_t off = lower ? lower_panel_offset(P) : upper_panel_offset(P, n_pad);
    const float2 *ph = Ph + off, *pl = Pl + off;
    const int kp1 = lower ? (P + 1) * PH / 2 : (n_pad - P * PH) / 2;
    const int kcol0 = lower ? 0 : P * PH;
    dsf ar[2][R], ai[2][R];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < R; ++c) { ar[q][c] = dsf{0.f, 0.f}; ai[q][c] = dsf{0.f, 0.f}; }
    const int per = (kp1 + NW - 1) / NW;
    const int a = warp * per, b = min(kp1, a + per);
    for (int kp = a; kp < b; ++kp) {
        const int64_t to = (int64_t)kp * (2 * PH) + 2 * lane;
        float2 th[2][2], tl[2][2];
        th[0][0] = ph[to]; th[0][1] = ph[to + 1]; th[1][0] = ph[to + 64]; th[1][1] = ph[to + 65];
        tl[0][0] = pl[to]; tl[0][1] = pl[to + 1]; tl[1][0] = pl[to + 64]; tl[1][1] = pl[to + 65];
        const int k0 = kcol0 + 2 * kp;
#pragma unroll
        for (int c = 0; c < R; ++c) {
            const int cc = s_col[c];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                float xrh = 0.f, xih = 0.f, xrl = 0.f, xil = 0.f;
                if (cc >= 0 && k0 + u < n) {
                    if (Xh) {  // pre-split operand: no FP64 instruction in the loop
                        const float2 vh = Xh[(int64_t)(k0 + u) * ldx + cc], vl = Xl[(int64_t)(k0 + u) * ldx + cc];
                        xrh = vh.x; xih = vh.y; xrl = vl.x; xil = vl.y;
                    } else {
                        const double2 xv = X[(int64_t)(k0 + u) * ldx + cc];
                        xrh = (float)xv.x; xih = (float)xv.y;
                        xrl = (float)(xv.x - (double)xrh); xil = (float)(xv.y - (double)xih);
                    }
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float2 h = th[q][u], l = tl[q][u];
                    // re += t.re x.re - t.im x.im ; im += t.re x.im + t.im x.re
                    ds_acc(ar[q][c], h.x, l.x, xrh, xrl);
                    ds_acc(ar[q][c], -h.y, -l.y, xih, xil);
                    ds_acc(ai[q][c], h.x, l.x, xih, xil);
                    ds_acc(ai[q][c], h.y, l.y, xrh, xrl);
                }
            }
        }
        // renormalise (fast two-sum) so that |lo| stays within an ulp of hi
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int c = 0; c < R; ++c) {
                ds_norm(ar[q][c]);
                ds_norm(ai[q][c]);
            }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < R; ++c) red[warp][lane + 32 * q][c] = make_double2(ds_val(ar[q][c]), ds_val(ai[q][c]));
    __syncthreads();
    for (int e = threadIdx.x; e < PH * R; e += NW * 32) {
        const int li = e / R, c = e % R, row = P * PH + li, cc = s_col[c];
        if (row >= n || cc < 0) continue;
        double2 y = make_double2(0.0, 0.0);
        for (int w = 0; w < NW; ++w) y = cadd(y, red[w][li][c]);
        const double2 xr = X[(int64_t)row * ldx + cc];
        cfms(y, s_z[c], xr);
        if (subtract) y = csub(B[(int64_t)row * ldb + cc], y);
        Y[(int64_t)row * ldy + cc] = y;
    }
}

// x = hi + lo as FP32 pairs for the listed columns (all if cols == nullptr):
// the only FP64 work of a double-single product, done once per element
// instead of once per row panel.
__global__ void split_ds_kernel(const double2 *__restrict__ X, int n, int64_t ldx, const int *__restrict__ cols,
                                int ncols, float2 *__restrict__ Xh, float2 *__restrict__ Xl) {
    const int t = blockIdx.x * 32 + (threadIdx.x & 31);
    if (t >= ncols) return;
    const int c = cols ? cols[t] : t;
    for (int i = threadIdx.x >> 5; i < n; i += blockDim.x >> 5) {
        const double2 v = X[(int64_t)i * ldx + c];
        const float hx = (float)v.x, hy = (float)v.y;
        Xh[(int64_t)i * ldx + c] = make_float2(hx, hy);
        Xl[(int64_t)i * ldx + c] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
    }
}

constexpr int RDS = 4, NW_DS = 8;
cudaError_t launch_trmv_ds(const float2 *Ph, const float2 *Pl, int n, int n_pad, int lower, const int *cols,
                           const double2 *zc, int ncols, const double2 *X, int64_t ldx, const double2 *B, int64_t ldb,
                           double2 *Y, int64_t ldy, int subtract, cudaStream_t s, float2 *Xh, float2 *Xl) {
    if (ncols <= 0) return cudaSuccess;
    if (Xh && Xl) {
        note_launch(); split_ds_kernel<<<(ncols + 31) / 32, 256, 0, s>>>(X, n, ldx, cols, ncols, Xh, Xl);
    } else {
        Xh = Xl = nullptr;
    }
    dim3 grid(n_pad / PH, (ncols + RDS - 1) / RDS);
    note_launch(); trmv_ds_kernel<RDS, NW_DS><<<grid, NW_DS * 32, 0, s>>>(Ph, Pl, n, n_pad, lower, cols, zc, ncols, X, Xh, Xl, ldx,
                                                                          B, ldb, Y, ldy, subtract);
    return cudaGetLastError();
}

// low FP32 plane: fl32(T - fl32(T)) in the same packed layout
__global__ void pack_lo_kernel(const double2 *__restrict__ P64, const float2 *__restrict__ P32, float2 *__restrict__ Plo,
                               int64_t cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        Plo[i] = make_float2((float)(P64[i].x - (double)P32[i].x), (float)(P64[i].y - (double)P32[i].y));
}
void launch_pack_lo(const double2 *P64, const float2 *P32, float2 *Plo, int64_t cnt, cudaStream_t s) {
    note_launch(); pack_lo_kernel<<<1184, 256, 0, s>>>(P64, P32, Plo, cnt);
}

// ------------------------------------------------------------------ norms
__global__ void sumsq_kernel(const double2 *__restrict__ a, int64_t cnt, double *out) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        s += a[i].x * a[i].x + a[i].y * a[i].y;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(out, s);
    }
}

cudaError_t launch_sumsq(const double2 *a, int64_t cnt, double *out, cudaStream_t s) {
    cudaMemsetAsync(out, 0, sizeof(double), s);
    note_launch(); sumsq_kernel<<<296, 256, 0, s>>>(a, cnt, out);
    return cudaGetLastError();
}

__global__ void extract_diag_kernel(const double2 *__restrict__ U, int n, int n_pad, double2 *__restrict__ d) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int P = i / PH, li = i % PH;
    d[i] = U[upper_panel_offset(P, n_pad) + (int64_t)(li >> 1) * (2 * PH) + 2 * li + (li & 1)];
}

cudaError_t launch_extract_diag(const double2 *U, int n, int n_pad, double2 *d, cudaStream_t s) {
    note_launch(); extract_diag_kernel<<<(n + 255) / 256, 256, 0, s>>>(U, n, n_pad, d);
    return cudaGetLastError();
}

}  // namespace pseudo
