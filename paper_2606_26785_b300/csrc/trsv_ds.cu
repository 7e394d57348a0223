// Multi-shift triangular solve in double-single arithmetic on the FP32 units:
// (T - z_c I) x_c = b_c or (T - z_c I)^H x_c = b_c for many columns at once,
// the R(z)^{-1} / R(z)^{-*} applications (Alg. 3, the inverse-Lanczos
// comparator) for the points that the FP32 solves cannot serve.
//
// FP64 runs at 1/64 of the FP32 rate on this part.  Here every number is an
// unevaluated sum hi + lo of two FP32 values (about 48 significant bits): T
// comes as its FP32 panels and the FP32 panels of T - fl32(T) (the same pair
// the double-single products use), a product of two such numbers keeps its
// leading part exactly (TwoProd: p = a b, e = fma(a, b, -p)), and every
// addition into an accumulator is exact in its leading part (TwoSum), with the
// rounding errors collected in the low word.  A complex multiply-add costs
// about 44 FP32 instructions against 4 FP64 FMAs at 1/64 rate: about six
// times the FP64 throughput at the same blocking.
//
// Blocking and data layout follow the CUDA-core solve of tri_kernels.cu: a CTA
// owns R right-hand sides and walks the 64-row panels (bottom-up for T,
// top-down for T^H); the warps split the off-diagonal contribution, sum it
// through shared memory, and solve the 64 x 64 shifted diagonal block with
// warp shuffles.  Solved values are kept per CTA in a compact copy already
// split into (hi, lo) pairs, so the inner loop touches no FP64 instruction;
// right-hand sides are read, and solutions written, as FP64.
#include "common.cuh"
#include "driver.h"
#include "internal.h"

namespace pseudo {

namespace {

struct __align__(16) dsc {
    float rh, rl, ih, il;  // complex double-single: (rh + rl) + i (ih + il)
};

__device__ __forceinline__ dsc ds_zero() { return dsc{0.f, 0.f, 0.f, 0.f}; }

__device__ __forceinline__ dsc ds_from(double2 v) {
    const float rh = (float)v.x, ih = (float)v.y;
    return dsc{rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih)};
}
__device__ __forceinline__ double2 ds_to(const dsc &a) {
    return make_double2((double)a.rh + (double)a.rl, (double)a.ih + (double)a.il);
}

// hi + lo += a * b exactly in the leading part (TwoProd + TwoSum); the low
// word collects the two rounding errors and the extra low-order term `low`
__device__ __forceinline__ void ds_acc(float &hi, float &lo, float a, float b, float low) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    const float s = hi + p;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += (e + pe) + low;
}

// acc += sgn * t * x for a complex double-single t = (th, tl) and x
__device__ __forceinline__ void ds_cfma(dsc &acc, float2 th, float2 tl, const dsc &x, float sgn) {
    const float ar = sgn * th.x, ai = sgn * th.y, alr = sgn * tl.x, ali = sgn * tl.y;
    // real: ar xr - ai xi (+ low: ar xrl + alr xr - ai xil - ali xi)
    const float lr = fmaf(ar, x.rl, fmaf(alr, x.rh, fmaf(-ai, x.il, -ali * x.ih)));
    ds_acc(acc.rh, acc.rl, ar, x.rh, lr);
    ds_acc(acc.rh, acc.rl, -ai, x.ih, 0.f);
    // imag: ar xi + ai xr (+ low: ar xil + alr xi + ai xrl + ali xr)
    const float li = fmaf(ar, x.il, fmaf(alr, x.ih, fmaf(ai, x.rl, ali * x.rh)));
    ds_acc(acc.ih, acc.il, ar, x.ih, li);
    ds_acc(acc.ih, acc.il, ai, x.rh, 0.f);
}

// a -= b (both double-single)
__device__ __forceinline__ void ds_csub(dsc &a, const dsc &b) {
    float s = a.rh - b.rh, bb = s - a.rh;
    float e = (a.rh - (s - bb)) + (-b.rh - bb);
    a.rh = s;
    a.rl += e - b.rl;
    s = a.ih - b.ih;
    bb = s - a.ih;
    e = (a.ih - (s - bb)) + (-b.ih - bb);
    a.ih = s;
    a.il += e - b.il;
}
// a += b
__device__ __forceinline__ void ds_cadd(dsc &a, const dsc &b) {
    dsc nb{-b.rh, -b.rl, -b.ih, -b.il};
    ds_csub(a, nb);
}

// product of two complex double-single numbers
__device__ __forceinline__ dsc ds_cmul(const dsc &a, const dsc &b) {
    dsc r = ds_zero();
    ds_cfma(r, make_float2(a.rh, a.ih), make_float2(a.rl, a.il), b, 1.f);
    return r;
}

__device__ __forceinline__ dsc ds_shfl(const dsc &v, int src) {
    return dsc{__shfl_sync(0xffffffffu, v.rh, src), __shfl_sync(0xffffffffu, v.rl, src),
               __shfl_sync(0xffffffffu, v.ih, src), __shfl_sync(0xffffffffu, v.il, src)};
}

}  // namespace

template <int R, int NW>
__global__ void __launch_bounds__(NW * 32)
trsv_ds_kernel(const float2 *__restrict__ Ph, const float2 *__restrict__ Pl, const double2 *__restrict__ Pd,
               int n, int n_pad, int lower, const int *__restrict__ cols, const double2 *__restrict__ zc,
               int ncols_host, const int *__restrict__ ncols_dev, double2 *X, int64_t ldx, dsc *xs_all) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dsc *red = reinterpret_cast<dsc *>(smem_raw);  // [NW][PH][R]
    dsc *s_dinv = red + NW * PH * R;               // [PH][R]
    __shared__ int s_col[R];
    __shared__ double2 s_z[R];

    const int ncols = ncols_dev ? *ncols_dev : ncols_host;
    const int g = blockIdx.x;
    if (g * R >= ncols) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < R) {
        const int pos = g * R + threadIdx.x;
        int c = -1;
        double2 z = make_double2(0.0, 0.0);
        if (pos < ncols) { c = cols ? cols[pos] : pos; z = zc[c]; }
        if (lower) z.y = -z.y;  // (T - zI)^H = T^H - conj(z) I
        s_col[threadIdx.x] = c;
        s_z[threadIdx.x] = z;
    }
    __syncthreads();
    dsc *xs = xs_all + (int64_t)g * n_pad * R;
    const int npan = n_pad / PH;

    for (int step = 0; step < npan; ++step) {
        const int P = lower ? step : npan - 1 - step;
        const int64_t poff = lower ? lower_panel_offset(P) : upper_panel_offset(P, n_pad);
        const float2 *ph = Ph + poff, *pl = Pl + poff;
        int kp0, kp1, kcol0;
        if (!lower) { kp0 = PH / 2; kp1 = (n_pad - P * PH) / 2; kcol0 = P * PH; }
        else { kp0 = 0; kp1 = P * PH / 2; kcol0 = 0; }

        dsc acc[2][R];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int c = 0; c < R; ++c) acc[q][c] = ds_zero();

        const int nk = kp1 - kp0;
        const int per = (nk + NW - 1) / NW;
        const int a = kp0 + warp * per;
        const int b = min(kp1, a + per);
        for (int kp = a; kp < b; ++kp) {
            const int64_t o = (int64_t)kp * (2 * PH) + 2 * lane;
            const float2 h00 = ph[o], h01 = ph[o + 1], h10 = ph[o + 64], h11 = ph[o + 65];
            const float2 l00 = pl[o], l01 = pl[o + 1], l10 = pl[o + 64], l11 = pl[o + 65];
            const dsc *x0 = xs + (int64_t)(kcol0 + 2 * kp) * R;
#pragma unroll
            for (int c = 0; c < R; ++c) {
                const dsc xa = x0[c], xb = x0[R + c];
                ds_cfma(acc[0][c], h00, l00, xa, 1.f);
                ds_cfma(acc[0][c], h01, l01, xb, 1.f);
                ds_cfma(acc[1][c], h10, l10, xa, 1.f);
                ds_cfma(acc[1][c], h11, l11, xb, 1.f);
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int c = 0; c < R; ++c) red[((warp * PH) + lane + 32 * q) * R + c] = acc[q][c];
        // 1 / (t_ii - z_c) for every row of the panel and column, in FP64 (PH R
        // values per panel), stored as double-single
        for (int e = threadIdx.x; e < PH * R; e += NW * 32) {
            const int li = e / R, c = e % R, row = P * PH + li;
            dsc d = ds_zero();
            if (row < n) {
                const int64_t dp = lower ? (int64_t)(P * 32 + (li >> 1)) : (int64_t)(li >> 1);
                const double2 t = Pd[poff + dp * (2 * PH) + 2 * li + (li & 1)];
                const double dr = t.x - s_z[c].x, di = t.y - s_z[c].y;
                const double m = dr * dr + di * di;
                d = ds_from(m > 0.0 ? make_double2(dr / m, -di / m) : make_double2(0.0, 0.0));
            }
            s_dinv[li * R + c] = d;
        }
        __syncthreads();

        constexpr int CPW = (R + NW - 1) / NW;
        const int c0 = warp * CPW;
        if (c0 < R) {
            dsc tot[2][CPW];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int row = P * PH + lane + 32 * q;
#pragma unroll
                for (int cc = 0; cc < CPW; ++cc) {
                    const int c = c0 + cc;
                    dsc bv = ds_zero();
                    if (c < R) {
                        if (row < n && s_col[c] >= 0) bv = ds_from(X[(int64_t)row * ldx + s_col[c]]);
                        dsc sum = ds_zero();
#pragma unroll
                        for (int w = 0; w < NW; ++w) ds_cadd(sum, red[((w * PH) + lane + 32 * q) * R + c]);
                        ds_csub(bv, sum);
                    }
                    tot[q][cc] = bv;
                }
            }
            if (!lower) {
#pragma unroll
                for (int q = 1; q >= 0; --q) {
                    for (int l = 31; l >= 0; --l) {
                        const int i = 32 * q + l;
                        const int64_t di = (int64_t)(i >> 1) * (2 * PH) + (i & 1);
                        const float2 h0 = ph[di + 2 * lane], h1 = ph[di + 2 * (lane + 32)];
                        const float2 l0 = pl[di + 2 * lane], l1 = pl[di + 2 * (lane + 32)];
#pragma unroll
                        for (int cc = 0; cc < CPW; ++cc) {
                            const int c = min(c0 + cc, R - 1);
                            const dsc xi = ds_shfl(ds_cmul(tot[q][cc], s_dinv[i * R + c]), l);
                            if (lane == l) tot[q][cc] = xi;
                            if (q == 1) {
                                ds_cfma(tot[0][cc], h0, l0, xi, -1.f);
                                if (lane < l) ds_cfma(tot[1][cc], h1, l1, xi, -1.f);
                            } else {
                                if (lane < l) ds_cfma(tot[0][cc], h0, l0, xi, -1.f);
                            }
                        }
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    for (int l = 0; l < 32; ++l) {
                        const int i = 32 * q + l;
                        const int64_t di = (int64_t)(P * 32 + (i >> 1)) * (2 * PH) + (i & 1);
                        const float2 h0 = ph[di + 2 * lane], h1 = ph[di + 2 * (lane + 32)];
                        const float2 l0 = pl[di + 2 * lane], l1 = pl[di + 2 * (lane + 32)];
#pragma unroll
                        for (int cc = 0; cc < CPW; ++cc) {
                            const int c = min(c0 + cc, R - 1);
                            const dsc xi = ds_shfl(ds_cmul(tot[q][cc], s_dinv[i * R + c]), l);
                            if (lane == l) tot[q][cc] = xi;
                            if (q == 0) {
                                if (lane > l) ds_cfma(tot[0][cc], h0, l0, xi, -1.f);
                                ds_cfma(tot[1][cc], h1, l1, xi, -1.f);
                            } else {
                                if (lane > l) ds_cfma(tot[1][cc], h1, l1, xi, -1.f);
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
                    const dsc v = row < n ? tot[q][cc] : ds_zero();
                    xs[(int64_t)row * R + c] = v;
                    if (row < n && s_col[c] >= 0) X[(int64_t)row * ldx + s_col[c]] = ds_to(v);
                }
            }
        }
        __syncthreads();
    }
}

namespace {
constexpr int RDS = 8, NW_DS = 8;

template <int R>
cudaError_t trsv_ds_launch(const float2 *Ph, const float2 *Pl, const double2 *Pd, int n, int n_pad, int lower,
                           const int *cols, const double2 *zc, int ncols, const int *ncols_dev, double2 *X,
                           int64_t ldx, void *xs, cudaStream_t s) {
    const size_t sm = sizeof(dsc) * (size_t)(NW_DS * PH * R + PH * R);
    static std::atomic<uint64_t> attr{0};
    smem_attr_once(trsv_ds_kernel<R, NW_DS>, (int)sm, attr);
    const int grid = (ncols + R - 1) / R;
    if (grid == 0) return cudaSuccess;
    note_launch();
    trsv_ds_kernel<R, NW_DS><<<grid, NW_DS * 32, sm, s>>>(Ph, Pl, Pd, n, n_pad, lower, cols, zc, ncols, ncols_dev, X,
                                                         ldx, (dsc *)xs);
    return cudaGetLastError();
}
}  // namespace

// Scratch of the double-single solve: one n_pad x 8 compact copy (16 bytes per
// element) per group of 8 columns; narrower groups of small launches fit in it.
size_t trsv_ds_scratch_bytes(int64_t n_pad, int64_t ncols) {
    const int64_t groups = (ncols + RDS - 1) / RDS;
    return (size_t)groups * n_pad * RDS * sizeof(dsc);
}

cudaError_t launch_trsv_ds(const pseudo_ctx *h, int lower, const int *cols, const double2 *zc, int ncols,
                           const int *ncols_dev, double2 *X, int64_t ldx, void *xs, cudaStream_t s) {
    const float2 *Ph = lower ? h->L32 : h->U32, *Pl = lower ? h->L32lo : h->U32lo;
    const double2 *Pd = lower ? h->L64 : h->U64;
    // a launch of few columns still spreads over the SMs (as the FP64 solve)
    if (ncols <= 296)
        return trsv_ds_launch<2>(Ph, Pl, Pd, h->n, h->n_pad, lower, cols, zc, ncols, ncols_dev, X, ldx, xs, s);
    return trsv_ds_launch<RDS>(Ph, Pl, Pd, h->n, h->n_pad, lower, cols, zc, ncols, ncols_dev, X, ldx, xs, s);
}

}  // namespace pseudo
