// Rectangular input, m >= 2n (SM2.2).  After the preliminary reduction the
// pencil is M(z) = M - zS with M = [T; B] (2n x n) and S = [I; 0]; here T and B
// are both upper triangular (the host reduction takes the Schur form of the
// top block, C_u = U T U^H, and the triangular factor of R_l U, so that the
// singular values are those of C - zI).  Unlike the square case, M(z) is not
// triangular, so every point needs its own QR factorisation M(z) = Q R(z)
// (Alg. 3, the triangular factor of eq. (triGen)); sigma_min(M(z)) =
// sigma_min(R(z)), and inverse Lanczos runs on R(z)^H R(z).
//
// B300 layout: each Lanczos slot owns its factor R(z) (packed upper triangle,
// column-major, FP64, the reciprocals of its diagonal stored in place of the
// diagonal) and a work copy of B for the factorisation.  A slot's
// factor is rebuilt only when the slot gets a new point (rect_qr_kernel:
// one CTA per such slot, Householder reflectors that pair row k of the top
// block with rows 0..k of the bottom one -- the bottom block's fill stays in
// its upper triangle, so the work is n^3/3 complex multiply-adds, not the
// 4n^3/3 of a dense 2n x n QR).  The two triangular solves of a Lanczos step
// (rect_solve_kernel) give each running slot one warp that walks its own
// factor; the right-hand side sits in shared memory (one n-vector per warp,
// which bounds n at RECT_N_MAX for a single warp in 227 KB).
#define RECT_N_MAX 14000
#include <algorithm>

#include "common.cuh"
#include "driver.h"
#include "internal.h"

namespace pseudo {

int rect_max_order() { return RECT_N_MAX; }
int64_t rect_packed_size(int n) { return (int64_t)n * (n + 1) / 2; }

// packed column-major upper triangle: (i, j), i <= j, at j (j + 1) / 2 + i
__device__ __forceinline__ int64_t up_idx(int i, int j) { return (int64_t)j * (j + 1) / 2 + i; }

// acc += conj(a) b in four fused multiply-adds
__device__ __forceinline__ void cfmac(double2 &acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

// acc -= conj(a) b
__device__ __forceinline__ void cfmsc(double2 &acc, double2 a, double2 b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

__device__ __forceinline__ double2 warp_sum_c(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

constexpr int QR_THREADS = 256, QR_WARPS = QR_THREADS / 32;
// up to this order a reflector step gives every remaining column a thread;
// above it a warp (measured: n = 150 runs 1.9x faster with threads, n = 600
// 1.35x faster with warps, whose column reads stay coalesced)
constexpr int QR_THREAD_COLUMNS_MAX = 256;

// Householder QR of M(z) = [T - zI; B] for the running slots whose factor is
// stale (Rz[c] != zslot[c]; NaN marks none).  Step k builds the reflector
// H = I - tau v v^H with H^H [alpha; x] = [beta; 0], alpha = R(k, k), x =
// column k of the bottom block (rows 0..k), beta = -sign(Re alpha) sqrt(|alpha|^2
// + |x|^2), tau = (beta - alpha) / beta, v = [1; x / (alpha - beta)], and
// applies H^H to columns k+1..n-1 of top row k and bottom rows 0..k (one
// thread or one warp per column).  Rows of
// the top block other than k take no part (their column-k entry is zero),
// and the bottom block keeps its upper-triangular support.  R(z) is the top
// block at the end.  Dynamic shared memory: n complex (the reflector).
__global__ void __launch_bounds__(QR_THREADS)
rect_qr_kernel(const double2 *__restrict__ M, int64_t ldm, int n, const int *__restrict__ cols, int ncols,
               const int *__restrict__ ncols_dev, const double2 *__restrict__ zslot, double2 *__restrict__ Rz,
               double2 *__restrict__ Rs, double2 *__restrict__ Bs) {
    extern __shared__ double2 vs[];
    __shared__ double red[QR_WARPS];
    __shared__ double2 s_tau;
    __shared__ int s_skip;
    const int nl = ncols_dev ? min(*ncols_dev, ncols) : ncols;
    const int p = blockIdx.x;
    if (p >= nl) return;
    const int c = cols ? cols[p] : p;
    const double2 z = zslot[c];
    {
        const double2 zr = Rz[c];
        if (zr.x == z.x && zr.y == z.y) return;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t psz = (int64_t)n * (n + 1) / 2;
    double2 *R = Rs + (int64_t)c * psz, *Bw = Bs + (int64_t)c * psz;
    for (int j = warp; j < n; j += QR_WARPS) {
        const double2 *mc = M + (int64_t)j * ldm;
        for (int i = lane; i <= j; i += 32) {
            double2 t = mc[i];
            if (i == j) { t.x -= z.x; t.y -= z.y; }
            R[up_idx(i, j)] = t;
            Bw[up_idx(i, j)] = mc[n + i];
        }
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        double sq = 0.0;
        for (int i = tid; i <= k; i += QR_THREADS) sq += cabs2(Bw[up_idx(i, k)]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) red[warp] = sq;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < QR_WARPS; ++w) t += red[w];
            const double2 alpha = R[up_idx(k, k)];
            if (t == 0.0) {
                s_skip = 1;
            } else {
                const double beta = -copysign(hypot(hypot(alpha.x, alpha.y), sqrt(t)), alpha.x);
                s_tau = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
                vs[k] = crecip(make_double2(alpha.x - beta, alpha.y));  // the scale of x, parked in vs[k]
                R[up_idx(k, k)] = make_double2(beta, 0.0);
                s_skip = 0;
            }
        }
        __syncthreads();
        if (s_skip) continue;  // uniform: the reflector is the identity
        const double2 scale = vs[k];
        __syncthreads();
        for (int i = tid; i <= k; i += QR_THREADS) vs[i] = cmul(scale, Bw[up_idx(i, k)]);
        __syncthreads();
        const double2 ctau = cconj(s_tau);
        if (n > QR_THREAD_COLUMNS_MAX) {
            // one warp per remaining column: coalesced reads of the column, and
            // its update while the column is still in L1
            for (int j = k + 1 + warp; j < n; j += QR_WARPS) {
                double2 *bc = Bw + up_idx(0, j);
                double2 w = make_double2(0.0, 0.0);
                for (int i = lane; i <= k; i += 32) cfmac(w, vs[i], bc[i]);
                w = warp_sum_c(w);
                double2 *rk = R + up_idx(k, j);
                w = cadd(w, *rk);
                const double2 tw = cmul(ctau, w);
                for (int i = lane; i <= k; i += 32) cfms(bc[i], tw, vs[i]);
                if (lane == 0) *rk = csub(*rk, tw);
            }
            __syncthreads();
            continue;
        }
        // small n: one thread per remaining column; it walks its own column
        // (contiguous in the packed layout) twice, the reflector coming from
        // shared memory as a broadcast, with no cross-lane reduction
        for (int j = k + 1 + tid; j < n; j += QR_THREADS) {
            double2 *bc = Bw + up_idx(0, j);
            double2 *rk = R + up_idx(k, j);
            double2 w0 = *rk, w1 = make_double2(0.0, 0.0), w2 = w1, w3 = w1;
            int i = 0;
            for (; i + 3 <= k; i += 4) {  // four partial sums: the thread's chain is the latency
                cfmac(w0, vs[i], bc[i]);
                cfmac(w1, vs[i + 1], bc[i + 1]);
                cfmac(w2, vs[i + 2], bc[i + 2]);
                cfmac(w3, vs[i + 3], bc[i + 3]);
            }
            for (; i <= k; ++i) cfmac(w0, vs[i], bc[i]);
            const double2 tw = cmul(ctau, cadd(cadd(w0, w1), cadd(w2, w3)));
            for (i = 0; i <= k; ++i) cfms(bc[i], tw, vs[i]);
            *rk = csub(*rk, tw);
        }
        __syncthreads();
    }
    // the solves divide by the diagonal: store its reciprocals in its place
    __syncthreads();
    for (int i = tid; i < n; i += QR_THREADS) R[up_idx(i, i)] = crecip(R[up_idx(i, i)]);
    if (tid == 0) Rz[c] = z;
}

constexpr int RS_WARPS = 4;  // warps (slots) per CTA, fewer for large n

// Dynamic shared memory a CTA of `kernel` may opt into: the device's opt-in
// limit less the kernel's static shared memory.
template <typename K>
static int smem_cap(K kernel) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 48 * 1024;
    return optin - (int)fa.sharedSizeBytes;
}

// Per running slot (one warp): x <- R^{-H} x (lower = 1) or x <- R^{-1} x
// (lower = 0) with the slot's own factor R(z); x is column c of X (leading
// dimension ldx), copied to shared memory for the solve.  Dynamic shared
// memory: (blockDim.x / 32) * n complex.
__global__ void __launch_bounds__(RS_WARPS * 32)
rect_solve_kernel(const double2 *__restrict__ Rs, int n, int lower, const int *__restrict__ cols, int ncols,
                  const int *__restrict__ ncols_dev, double2 *X, int64_t ldx) {
    extern __shared__ double2 ys[];
    const int nl = ncols_dev ? min(*ncols_dev, ncols) : ncols;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * (int)(blockDim.x >> 5) + warp;
    if (p >= nl) return;  // no block-wide barrier below
    const int c = cols ? cols[p] : p;
    const double2 *R = Rs + (int64_t)c * ((int64_t)n * (n + 1) / 2);
    double2 *y = ys + (int64_t)warp * n;
    for (int i = lane; i < n; i += 32) y[i] = X[(int64_t)i * ldx + c];
    __syncwarp();
    if (lower) {
        // R^H y = x: y_i = (x_i - sum_{j<i} conj(R(j, i)) y_j) conj(1 / R(i, i)),
        // in blocks of 32 rows, lane l owning row i0 + l: first the part of its
        // sum over the rows solved before the block (its own column of R,
        // walked in order), then the 32 x 32 diagonal block by broadcasts
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            const double2 *col = R + up_idx(0, i < n ? i : i0);
            double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
            if (i < n) {
                int j = 0;
                for (; j + 1 < i0; j += 2) {
                    cfmac(s0, col[j], y[j]);
                    cfmac(s1, col[j + 1], y[j + 1]);
                }
                if (j < i0) cfmac(s0, col[j], y[j]);
            }
            double2 yi = i < n ? csub(y[i], cadd(s0, s1)) : make_double2(0.0, 0.0);
            const int tb = min(32, n - i0);
            for (int t = 0; t < tb; ++t) {
                if (lane == t) yi = cmulc(col[i], yi);  // conj(1 / R(i, i)) y_i
                const double2 yt = shfl_c(yi, t);
                if (lane > t && i < n) cfmsc(yi, col[i0 + t], yt);
            }
            if (i < n) y[i] = yi;
            __syncwarp();
        }
    } else {
        // R w = y: w_i = y_i (1 / R(i, i)), then y_j -= R(j, i) w_i for j < i
        for (int i = n - 1; i >= 0; --i) {
            const double2 *col = R + up_idx(0, i);
            const double2 wi = cmul(y[i], col[i]);
            for (int j = lane; j < i; j += 32) cfms(y[j], col[j], wi);
            __syncwarp();
            if (lane == 0) y[i] = wi;
            __syncwarp();
        }
    }
    for (int i = lane; i < n; i += 32) X[(int64_t)i * ldx + c] = y[i];
}

__global__ void add_cols_kernel(double2 *__restrict__ A, const double2 *__restrict__ B, int64_t cnt) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < cnt) A[t] = cadd(A[t], B[t]);
}

cudaError_t launch_rect_qr(const pseudo_ctx *h, const int *cols, int ncols, const int *ncols_dev,
                           const double2 *zslot, double2 *Rz, double2 *Rs, double2 *Bs, cudaStream_t s) {
    if (ncols <= 0) return cudaSuccess;
    const int n = h->n;
    const size_t sm = (size_t)n * sizeof(double2);
    static const int cap = smem_cap(rect_qr_kernel);
    if (sm > (size_t)cap) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> attr{0};
    smem_attr_once(rect_qr_kernel, cap, attr);
    note_launch();
    rect_qr_kernel<<<ncols, QR_THREADS, sm, s>>>(h->M64, 2 * (int64_t)n, n, cols, ncols, ncols_dev, zslot, Rz, Rs, Bs);
    return cudaGetLastError();
}

cudaError_t launch_rect_solve(const pseudo_ctx *h, const double2 *Rs, int lower, const int *cols, int ncols,
                              const int *ncols_dev, double2 *X, int64_t ldx, cudaStream_t s) {
    if (ncols <= 0) return cudaSuccess;
    const int n = h->n;
    static const int cap = smem_cap(rect_solve_kernel);
    const int wpb = (int)std::max<int64_t>(1, std::min<int64_t>(RS_WARPS, cap / ((int64_t)n * 16)));
    const size_t sm = (size_t)wpb * n * sizeof(double2);
    if (sm > (size_t)cap) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> attr{0};
    smem_attr_once(rect_solve_kernel, cap, attr);
    note_launch();
    rect_solve_kernel<<<(ncols + wpb - 1) / wpb, wpb * 32, sm, s>>>(Rs, n, lower, cols, ncols, ncols_dev, X, ldx);
    return cudaGetLastError();
}

void launch_add_cols(double2 *A, const double2 *B, int64_t cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    note_launch();
    add_cols_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(A, B, cnt);
}

// Y = M(z) x for the columns of X (Y: 2n rows, leading dimension ldy, the top
// block first) and, with NX non-null, NX = M(z)^H Y = (T - zI)^H Y_top +
// B^H Y_bot, with the FP64 panel kernels (B's products take no shift); Tb is
// n x ldx scratch.  ncols_dev as in trmv_hp.
cudaError_t rect_normal_product(pseudo_ctx *h, const double2 *zc, int ncols,
                                const int *ncols_dev, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                                double2 *NX, double2 *Tb, cudaStream_t s) {
    const int n = h->n, np = h->n_pad;
    double2 *Yt = Y, *Yb = Y + (int64_t)n * ldy;
    cudaError_t e = launch_trmv64(h->U64, n, np, 0, nullptr, zc, ncols, ncols_dev, X, ldx, nullptr, ldx, Yt, ldy, 0, s);
    if (e == cudaSuccess)
        e = launch_trmv64(h->BU64, n, np, 0, nullptr, nullptr, ncols, ncols_dev, X, ldx, nullptr, ldx, Yb, ldy, 0, s);
    if (e != cudaSuccess || !NX) return e;
    e = launch_trmv64(h->L64, n, np, 1, nullptr, zc, ncols, ncols_dev, Yt, ldy, nullptr, ldy, NX, ldx, 0, s);
    if (e == cudaSuccess)
        e = launch_trmv64(h->BL64, n, np, 1, nullptr, nullptr, ncols, ncols_dev, Yb, ldy, nullptr, ldy, Tb, ldx, 0, s);
    if (e != cudaSuccess) return e;
    launch_add_cols(NX, Tb, (int64_t)n * ldx, s);
    return cudaGetLastError();
}

}  // namespace pseudo
