// Shifted triangular products Y = (T - z_c I)^{op} X or Y = B - (T - z_c I)^{op} X
// to about 2^-46 relative accuracy on the tensor cores: the refinement
// residuals of mixed precision (mv_M in Table 2).
//
// Exact-accumulation splitting.  Each row i of A'' (the real form of T, see
// below) is scaled by 2^-e_i and each column c of X by 2^-f_c so that all
// entries lie in (-1, 1); then every entry v is written as
//     v = sum_{s<7} alpha_s 2^(-7-8s) + r,   alpha_s integers, |alpha_s| <= 129,
// and the alpha_s are exact bf16 values.  A product of two slices is an
// integer below 2^14.02, so FP32 sums of up to 7 * 128 such products (the
// slice pairs of one level L = s + t over 128 terms) are exact.  The MMA
// (kind::f16, bf16 in, FP32 accumulate) keeps one TMEM accumulator per level
// L = 0..6 (28 slice pairs); every 128 real terms the accumulators are read
// out and added, scaled by 2^(-14-8L), into a double-single sum per output.
// The dropped pairs (L >= 7) and the remainders are below 2^-55 per term.
//
// Complex as real: A'' = [[Re T, -Im T], [Im T, Re T]] (128 real rows = 64
// complex rows: first the real parts, then the imaginary parts) and
// B'' = [Re X; Im X], so A'' B'' = [Re; Im] of T X.  A'' slices are built once
// at handle creation, in the byte image the MMA reads (no-swizzle K-major core
// matrices), one image per (row tile, chunk of 16 complex columns); the X
// slices are built per call in the same form, per (column tile, chunk).
#include <cmath>

#include <cuda_bf16.h>

#include "common.cuh"
#include "driver.h"
#include "internal.h"
#include "tc.cuh"

namespace pseudo {

namespace {
constexpr int OZ_NS = 7;                 // slices per operand, levels 0..6
constexpr int OZ_CR = 64;                // complex rows per tile
constexpr int OZ_MR = 2 * OZ_CR;         // real rows (MMA M)
constexpr int OZ_NC = 64;                // complex columns per tile (MMA N)
constexpr int OZ_KC = 8;                 // complex K per chunk
constexpr int OZ_KR = 2 * OZ_KC;         // real K per chunk (one MMA k-step of 16)
constexpr int OZ_SEG = 128 / OZ_KR;      // chunks per exact segment (128 real terms)
constexpr int OZ_NSTG = 4;               // ring of chunk stages in shared memory
constexpr int OZ_TPC = 64 / OZ_KC;       // chunks per 64 complex columns
constexpr int OZ_A_SLICE = OZ_MR * OZ_KR;            // bf16 elements
constexpr int OZ_B_SLICE = OZ_NC * OZ_KR;
constexpr int OZ_A_IMG = OZ_NS * OZ_A_SLICE;         // 14336 elements, 28 KB
constexpr int OZ_B_IMG = OZ_NS * OZ_B_SLICE;         // 7168 elements, 14 KB
#ifndef OZ_GR
#define OZ_GR 8  // row tiles per group of the tile order (see trmv_oz_kernel)
#endif
constexpr int OZ_TH = 256;  // two warpgroups: each TMEM lane quarter is read by two warps,
                             // one per half of the output columns

// element index of (row, k) in a bf16 core-matrix tile with R rows
__host__ __device__ __forceinline__ int cm16(int row, int k, int R) {
    return (((k >> 3) * (R >> 3) + (row >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}
__host__ __device__ __forceinline__ int64_t nchunks(int n_pad) { return n_pad / OZ_KC; }
// chunk range of row tile I: upper product uses complex columns >= 64 I,
// the lower (T^H) product columns < 64 I + 64
__host__ __device__ __forceinline__ void chunk_range(int I, int n_pad, int lower, int &c0, int &c1) {
    if (!lower) { c0 = OZ_TPC * I; c1 = (int)nchunks(n_pad); }
    else { c0 = 0; c1 = OZ_TPC * (I + 1); }
}
// first image of row tile I in the packed A slices
__host__ __device__ __forceinline__ int64_t a_tile_base(int64_t I, int64_t n_pad, int lower) {
    return lower ? (OZ_TPC / 2) * I * (I + 1) : I * nchunks((int)n_pad) - (OZ_TPC / 2) * I * (I - 1);
}

// alpha_s of v (|v| < 1) by repeated rounding of the exact remainder kept as
// a pair of FP32 numbers
__device__ __forceinline__ void slices7(float ph, float pl, float (&a)[OZ_NS]) {
#pragma unroll
    for (int s = 0; s < OZ_NS; ++s) {
        const float sc = ldexpf(1.f, 7 + 8 * s);
        const float q = rintf(ph * sc);
        ph = fmaf(-q, 1.f / sc, ph);  // exact: q / sc is within half a unit of ph's leading bits
        const float t = ph + pl;       // renormalise the remainder pair (TwoSum)
        const float bb = t - ph;
        pl = (ph - (t - bb)) + (pl - bb);
        ph = t;
        a[s] = q;
    }
}
}  // namespace

int64_t oz_a_elems(int n_pad) {
    const int64_t T = n_pad / OZ_CR;
    return a_tile_base(T, n_pad, 0) * OZ_A_IMG;  // the same total for both directions
}
size_t oz_scratch_bytes(int n_pad, int64_t ncols) {
    const int64_t ct = (ncols + OZ_NC - 1) / OZ_NC;
    return 256 + (size_t)ct * OZ_NC * sizeof(int) + (size_t)ct * nchunks(n_pad) * OZ_B_IMG * sizeof(__nv_bfloat16);
}

// ---------------------------------------------------------------- packing
// per complex row i: e_i with max_k |Re|, |Im| of row i of T (or T^H) < 2^e_i
__global__ void oz_rowexp_kernel(const double2 *__restrict__ T, int64_t ldT, int n, int n_pad, int lower,
                                 int *__restrict__ ex) {
    const int i = blockIdx.x;
    double m = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        if (i < n) {
            if (!lower && k >= i) v = T[(int64_t)k * ldT + i];
            if (lower && k <= i) v = T[(int64_t)i * ldT + k];
        }
        m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
    }
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        m = fmax(m, red[0]);
        int e = 0;
        if (m > 0.0) { frexp(m, &e); }  // m < 2^e
        ex[i] = e;
    }
}

__global__ void oz_pack_a_kernel(const double2 *__restrict__ T, int64_t ldT, int n, int n_pad, int lower,
                                 const int *__restrict__ ex, __nv_bfloat16 *__restrict__ out, int64_t total) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t img = e / OZ_A_IMG;
    const int w = (int)(e % OZ_A_IMG);
    const int s = w / OZ_A_SLICE, ww = w % OZ_A_SLICE;
    // invert cm16 for R = 128 rows
    const int cmi = ww >> 6, r7 = (ww >> 3) & 7, k7 = ww & 7;
    const int kb = cmi / (OZ_MR / 8), rb = cmi % (OZ_MR / 8);
    const int r = rb * 8 + r7, kk = kb * 8 + k7;
    // tile I and chunk of this image
    const int NT = n_pad / OZ_CR;
    int I = 0;
    {
        int lo = 0, hi = NT - 1;
        while (lo < hi) {  // largest I with a_tile_base(I) <= img
            const int mid = (lo + hi + 1) / 2;
            if (a_tile_base(mid, n_pad, lower) <= img) lo = mid; else hi = mid - 1;
        }
        I = lo;
    }
    int c0, c1;
    chunk_range(I, n_pad, lower, c0, c1);
    const int chunk = c0 + (int)(img - a_tile_base(I, n_pad, lower));
    const int i = I * OZ_CR + (r % OZ_CR), part = r / OZ_CR;
    const int k = chunk * OZ_KC + (kk % OZ_KC), kpart = kk / OZ_KC;
    double2 t = make_double2(0.0, 0.0);  // element (i, k) of T (upper) or T^H (lower)
    if (i < n && k < n) {
        if (!lower && k >= i) t = T[(int64_t)k * ldT + i];
        if (lower && k <= i) { t = T[(int64_t)i * ldT + k]; t.y = -t.y; }
    }
    // [[Re, -Im], [Im, Re]]
    const double v = part == 0 ? (kpart == 0 ? t.x : -t.y) : (kpart == 0 ? t.y : t.x);
    const double sv = i < n ? ldexp(v, -ex[i]) : 0.0;
    const float ph = (float)sv, pl = (float)(sv - (double)ph);
    float a[OZ_NS];
    slices7(ph, pl, a);
    float pick = a[0];
#pragma unroll
    for (int q = 1; q < OZ_NS; ++q)
        if (q == s) pick = a[q];
    out[e] = __float2bfloat16_rn(pick);
}

void launch_pack_oz(const double2 *T, int64_t ldT, int n, int n_pad, void *AUv, void *ALv, int *exU, int *exL,
                    cudaStream_t s) {
    __nv_bfloat16 *AU = (__nv_bfloat16 *)AUv, *AL = (__nv_bfloat16 *)ALv;
    note_launch(); oz_rowexp_kernel<<<n_pad, 256, 0, s>>>(T, ldT, n, n_pad, 0, exU);
    note_launch(); oz_rowexp_kernel<<<n_pad, 256, 0, s>>>(T, ldT, n, n_pad, 1, exL);
    const int64_t tot = oz_a_elems(n_pad);
    const unsigned bl = (unsigned)((tot + 255) / 256);
    note_launch(); oz_pack_a_kernel<<<bl, 256, 0, s>>>(T, ldT, n, n_pad, 0, exU, AU, tot);
    note_launch(); oz_pack_a_kernel<<<bl, 256, 0, s>>>(T, ldT, n, n_pad, 1, exL, AL, tot);
}

// ------------------------------------------------------------ X slicing
// f_p for listed column p: max_k |Re|, |Im| of column cols[p] < 2^f_p
__global__ void oz_colexp_kernel(const double2 *__restrict__ X, int n, int64_t ldx, const int *__restrict__ cols,
                                 int ncols, const int *__restrict__ ncols_dev, int *__restrict__ fx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    const int nl = ncols_dev ? min(*ncols_dev, ncols) : ncols;  // live columns
    const int c = p < nl ? (cols ? cols[p] : p) : -1;
    double m = 0.0;
    if (c >= 0)
        for (int i = warp; i < n; i += nw) {
            const double2 v = X[(int64_t)i * ldx + c];
            m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
        }
    __shared__ double red[32][33];
    red[warp][lane] = m;
    __syncthreads();
    if (warp == 0) {
        for (int w = 1; w < nw; ++w) m = fmax(m, red[w][lane]);
        int e = 0;
        if (m > 0.0) frexp(m, &e);
        if (p < ncols) fx[p] = e;
    }
}

// B'' slice images: one thread per (column tile, chunk, column j, group of 8
// real K entries), so that every slice is written as one 16-byte core-matrix
// row (8 consecutive bf16) and a warp reads 32 consecutive columns of X.
__global__ void oz_slice_b_kernel(const double2 *__restrict__ X, int n, int n_pad, int64_t ldx,
                                  const int *__restrict__ cols, int ncols, const int *__restrict__ ncols_dev,
                                  const int *__restrict__ fx, __nv_bfloat16 *__restrict__ img) {
    const int64_t NCH = nchunks(n_pad);
    const int nl = ncols_dev ? min(*ncols_dev, ncols) : ncols;  // live columns; the layout follows ncols
    const int64_t tiles = (nl + OZ_NC - 1) / OZ_NC;
    constexpr int KG = OZ_KR / 8;  // groups of 8 real K entries: real parts first, then imaginary parts
    const int64_t total = tiles * NCH * OZ_NC * KG;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(w % OZ_NC);
        const int kg = (int)((w / OZ_NC) % KG);
        const int64_t tc_ = w / ((int64_t)OZ_NC * KG);  // tile * NCH + chunk
        const int64_t ct = tc_ / NCH, ch = tc_ % NCH;
        const int p = (int)(ct * OZ_NC + j);
        const int part = kg / (KG / 2), kb = (kg % (KG / 2)) * 8;
        const bool live = p < nl;
        const int c = live ? (cols ? cols[p] : p) : 0;
        const int f = live ? fx[p] : 0;
        float a[8][OZ_NS];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = (int)(ch * OZ_KC) + kb + e;
            double v = 0.0;
            if (live && k < n) {
                const double2 x = X[(int64_t)k * ldx + c];
                v = part ? x.y : x.x;
            }
            const double sv = ldexp(v, -f);
            const float ph = (float)sv, pl = (float)(sv - (double)ph);
            slices7(ph, pl, a[e]);
        }
        __nv_bfloat16 *base = img + tc_ * OZ_B_IMG + cm16(j, kg * 8, OZ_NC);
#pragma unroll
        for (int s = 0; s < OZ_NS; ++s) {
            __align__(16) __nv_bfloat16 h[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) h[e] = __float2bfloat16_rn(a[e][s]);
            *reinterpret_cast<uint4 *>(base + s * OZ_B_SLICE) = *reinterpret_cast<const uint4 *>(h);
        }
    }
}

// ------------------------------------------------------------ the product
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float v) {
    const float t = hi + v;
    const float bb = t - hi;
    lo += (hi - (t - bb)) + (v - bb);
    hi = t;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

struct OzSmem {
    static constexpr size_t stage = (size_t)(OZ_A_IMG + OZ_B_IMG) * sizeof(__nv_bfloat16);  // 42 KB
    static constexpr size_t bytes = OZ_NSTG * stage + 128;
};

__global__ void __launch_bounds__(OZ_TH, 1)
trmv_oz_kernel(const __nv_bfloat16 *__restrict__ Apack, const int *__restrict__ ex, const __nv_bfloat16 *__restrict__ Bimg,
               const int *__restrict__ fx, int n, int n_pad, int lower, const int *__restrict__ cols,
               const double2 *__restrict__ zc, int ncols, const int *__restrict__ ncols_dev,
               const double2 *__restrict__ X, int64_t ldx, const double2 *__restrict__ B, int64_t ldb,
               double2 *__restrict__ Y, int64_t ldy, int subtract, int *err, uint64_t wait_ns) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_ld[OZ_NSTG], bar_mma[OZ_NSTG];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int NT = n_pad / OZ_CR;
    // Tile order: groups of OZ_GR row tiles, column tiles outer and row tiles
    // inner within a group, so that the CTAs resident at one time share a few
    // A slice streams (row tiles) and a few X slice streams (column tiles) in
    // L2 instead of every CTA of a row tile streaming its own X slices from
    // DRAM; groups run heaviest first (upper products are longest at the top).
    const int tiles = (ncols + OZ_NC - 1) / OZ_NC;
    const int64_t lin = blockIdx.x;
    const int64_t grp = lin / ((int64_t)OZ_GR * tiles);
    const int rows_in = min(OZ_GR, NT - (int)grp * OZ_GR);
    const int64_t w_in = lin - grp * OZ_GR * tiles;
    const int iy = (int)grp * OZ_GR + (int)(w_in % rows_in);
    const int ct = (int)(w_in / rows_in);
    // with a device column count the grid covers ncols (an upper bound) and
    // the tiles past the live columns leave at once
    const int nl = ncols_dev ? min(*ncols_dev, ncols) : ncols;
    if (ct * OZ_NC >= nl) return;
    const int I = lower ? NT - 1 - iy : iy;
    int c0, c1;
    chunk_range(I, n_pad, lower, c0, c1);
    const int nch = c1 - c0;
    unsigned char *base = smem_raw + ((128 - (tc::smem_u32(smem_raw) & 127)) & 127);
    const int64_t NCH = nchunks(n_pad);
    const __nv_bfloat16 *Ap = Apack + a_tile_base(I, n_pad, lower) * OZ_A_IMG;
    const __nv_bfloat16 *Bp = Bimg + ((int64_t)ct * NCH + c0) * OZ_B_IMG;

    if (tid == 0) {
        for (int i = 0; i < OZ_NSTG; ++i) { tc::mbar_init(&bar_ld[i], 1); tc::mbar_init(&bar_mma[i], 1); }
        tc::mbar_fence_init();
        s_abort = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;
    constexpr uint32_t idesc = idesc_bf16(OZ_MR, OZ_NC);
    constexpr uint32_t LBO_A = (OZ_MR / 8) * 128, LBO_B = (OZ_NC / 8) * 128;
    constexpr uint32_t STAGE = (uint32_t)OzSmem::stage;
    const uint32_t s0 = tc::smem_u32(base);

    constexpr int HC = OZ_NC / 2;              // output columns per thread
    const int lq = warp & 3, hc = warp >> 2;    // TMEM lane quarter, column half
    const int rr = lq * 32 + (tid & 31);        // real row of the tile (TMEM lane)
    float hi[HC], lo[HC];
#pragma unroll
    for (int j = 0; j < HC; ++j) { hi[j] = 0.f; lo[j] = 0.f; }

    auto issue_load = [&](int q) {
        const int st = q % OZ_NSTG;
        tc::mbar_expect_tx(&bar_ld[st], (uint32_t)OzSmem::stage);
        unsigned char *dst = base + st * OzSmem::stage;
        tc::bulk_g2s(dst, Ap + (int64_t)q * OZ_A_IMG, OZ_A_IMG * 2, &bar_ld[st]);
        tc::bulk_g2s(dst + OZ_A_IMG * 2, Bp + (int64_t)q * OZ_B_IMG, OZ_B_IMG * 2, &bar_ld[st]);
    };
    int ld_pending = -1, mma_last = -1;
    // chunks 0 .. NSTG-2 in flight before the first MMA; chunk q + NSTG - 1 is
    // loaded into the stage of chunk q - 1 once its MMAs are done
    if (tid == 0)
        for (int q = 0; q < OZ_NSTG - 1 && q < nch; ++q) { issue_load(q); ld_pending = q; }
    for (int q = 0; q < nch; ++q) {
        const int st = q % OZ_NSTG;
        if (tid == 0 && !s_abort) {
            if (!tc::mbar_wait(&bar_ld[st], (q / OZ_NSTG) & 1, wait_ns)) {
                s_abort = 1;
            } else {
                tc::tc_fence_after();
                const uint32_t a0 = s0 + st * STAGE, b0 = a0 + OZ_A_IMG * 2;
                const bool seg_first = (q % OZ_SEG) == 0;
                // one descriptor per operand stage; a slice is a fixed offset (the
                // start-address field holds smem byte address >> 4 and cannot carry)
                const uint64_t da0 = tc::smem_desc(a0, LBO_A, 128), db0 = tc::smem_desc(b0, LBO_B, 128);
                constexpr uint64_t AS = (OZ_A_SLICE * 2) >> 4, BS = (OZ_B_SLICE * 2) >> 4;
                static_assert(OZ_KR == 16, "one MMA k-step per chunk");
                // A slice outer, level inner: consecutive MMAs go to different
                // level accumulators and do not wait on each other
#pragma unroll
                for (int sa = 0; sa < OZ_NS; ++sa) {
#pragma unroll
                    for (int L = sa; L < OZ_NS; ++L)
                        mma_bf16(tmem + L * OZ_NC, da0 + sa * AS, db0 + (L - sa) * BS, idesc,
                                 (seg_first && sa == 0) ? 0u : 1u);
                }
                tc::mma_commit(&bar_mma[st]);
                mma_last = q;
                const int qn = q + OZ_NSTG - 1;
                if (qn < nch) {
                    if (q >= 1 && !tc::mbar_wait(&bar_mma[(q - 1) % OZ_NSTG], ((q - 1) / OZ_NSTG) & 1, wait_ns)) {
                        s_abort = 1;
                    } else {
                        issue_load(qn);
                        ld_pending = qn;
                    }
                }
            }
        }
        // end of an exact segment: fold the level sums into the double-single totals
        if ((q % OZ_SEG) == OZ_SEG - 1 || q == nch - 1) {
            if (tid == 0 && !s_abort && !tc::mbar_wait(&bar_mma[st], (q / OZ_NSTG) & 1, wait_ns)) s_abort = 1;
            __syncthreads();
            if (s_abort) break;
            tc::tc_fence_after();
#pragma unroll 1
            for (int L = 0; L < OZ_NS; ++L) {
                const float sc = ldexpf(1.f, -14 - 8 * L);
#pragma unroll
                for (int h = 0; h < HC / 16; ++h) {
                    float d[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + L * OZ_NC + hc * HC + h * 16, d);
                    if (L < 5) {
#pragma unroll
                        for (int u = 0; u < 16; ++u) two_sum_acc(hi[h * 16 + u], lo[h * 16 + u], d[u] * sc);
                    } else {
                        // a level-L segment sum is below 2^(9 - 8L) of the scale, so
                        // levels 5 and 6 (< 2^-31) can go into the low word with a
                        // plain FP32 add (rounding < 2^-55); levels up to 4 cannot
#pragma unroll
                        for (int u = 0; u < 16; ++u) lo[h * 16 + u] = fmaf(d[u], sc, lo[h * 16 + u]);
                    }
                }
            }
            tc::tc_fence_before();
            __syncthreads();
        }
    }
    // ---- epilogue: scale, shift, subtract, store (real row tid: part = tid / 64).
    // The stage buffers are free now; the sums go through them so that the
    // per-column loop below needs no register-resident arrays.
    if (!s_abort) {
        double *sums = reinterpret_cast<double *>(base);  // [OZ_NC][OZ_MR]
#pragma unroll
        for (int j = 0; j < HC; ++j) sums[(hc * HC + j) * OZ_MR + rr] = (double)hi[j] + (double)lo[j];
        const int part = rr / OZ_CR, i = I * OZ_CR + (rr % OZ_CR);
        if (i < n) {
            const int e_i = ex[i];
            const int jmax = min(HC, nl - ct * OZ_NC - hc * HC);
            for (int jj = 0; jj < jmax; ++jj) {
                const int j = hc * HC + jj;
                const int p = ct * OZ_NC + j;
                const int c = cols ? cols[p] : p;
                double y = ldexp(sums[j * OZ_MR + rr], e_i + fx[p]);
                const double2 x = X[(int64_t)i * ldx + c];
                if (zc) {
                    const double2 z = zc[c];
                    if (!lower) y -= part == 0 ? z.x * x.x - z.y * x.y : z.x * x.y + z.y * x.x;
                    else y -= part == 0 ? z.x * x.x + z.y * x.y : z.x * x.y - z.y * x.x;
                }
                double *yo = reinterpret_cast<double *>(Y + (int64_t)i * ldy + c) + part;
                if (subtract) *yo = reinterpret_cast<const double *>(B + (int64_t)i * ldb + c)[part] - y;
                else *yo = y;
            }
        }
    }
    if (tid == 0 && s_abort) {
        // loads run at most OZ_NSTG - 1 chunks ahead of the MMAs and a stage is
        // reloaded only after its MMAs are done: every copy still in flight is
        // one of the last OZ_NSTG - 1 issued, on a stage not re-armed since
        for (int q = ld_pending - OZ_NSTG + 2 < 0 ? 0 : ld_pending - OZ_NSTG + 2; q <= ld_pending; ++q)
            tc::mbar_wait(&bar_ld[q % OZ_NSTG], (q / OZ_NSTG) & 1, 100000000ull);
        if (mma_last >= 0) tc::mbar_wait(&bar_mma[mma_last % OZ_NSTG], (mma_last / OZ_NSTG) & 1, 100000000ull);
        atomicExch(err, 1);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

cudaError_t launch_trmv_oz(const pseudo_ctx *h, int lower, const int *cols, const double2 *zc, int ncols,
                           const double2 *X, int64_t ldx, const double2 *B, int64_t ldb, double2 *Y, int64_t ldy,
                           int subtract, void *scratch, cudaStream_t s, const int *ncols_dev) {
    if (ncols <= 0) return cudaSuccess;
    static std::atomic<uint64_t> attr{0};
    smem_attr_once(trmv_oz_kernel, (int)OzSmem::bytes, attr);
    const int n = h->n, n_pad = h->n_pad;
    char *p = (char *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
    const int64_t tiles = (ncols + OZ_NC - 1) / OZ_NC;
    int *fx = (int *)p;
    __nv_bfloat16 *img = (__nv_bfloat16 *)(p + ((tiles * OZ_NC * sizeof(int) + 255) & ~(size_t)255));
    note_launch(); oz_colexp_kernel<<<(ncols + 31) / 32, 256, 0, s>>>(X, n, ldx, cols, ncols, ncols_dev, fx);
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    note_launch(); oz_slice_b_kernel<<<nsm * 8, 256, 0, s>>>(X, n, n_pad, ldx, cols, ncols, ncols_dev, fx, img);
    const unsigned grid = (unsigned)(tiles * (n_pad / OZ_CR));
    note_launch();
    trmv_oz_kernel<<<grid, OZ_TH, OzSmem::bytes, s>>>((const __nv_bfloat16 *)(lower ? h->ozA_L : h->ozA_U), lower ? h->ozE_L : h->ozE_U, img, fx,
                                                      n, n_pad, lower, cols, zc, ncols, ncols_dev, X, ldx, B, ldb,
                                                      Y, ldy, subtract, h->dev_err, h->wait_ns);
    return cudaGetLastError();
}

}  // namespace pseudo
