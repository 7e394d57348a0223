// Kernels of the shift-batched LOBPCG-SVD refinement (Alg. SM1.2) applied to
// C = R(z)^{-*} = (T - zI)^{-H} for the largest singular triplets (sigma_min
// of T - zI is 1/xi_1).  Batch item b is one refined grid point; its blocks
// live in row-major n x (nitems * 3r) arrays S = [X W P] and CS = [CX CW CP]
// at column offset b * 3r.  The solves run through the multi-shift
// triangular kernels; this file holds the per-item small dense work and the
// column plumbing around it.
#include "common.cuh"
#include "internal.h"
#include "lobpcg.h"
#include "smalldense.cuh"

namespace pseudo {

constexpr int LB_THREADS = 256;

// Column-scaled Cholesky of the Gram A (m x m, in place) with a shifted retry
// (shifted CholeskyQR, Fukaya et al.) when a pivot fails.  Zero columns get a
// unit pivot.  Leaves the upper factor R (A_in = R^H R up to the shift) in A.
static __device__ void scaled_cholesky(double2 *A, double2 *Acopy, int m, double *d) {
    const int tid = threadIdx.x;
    for (int e = tid; e < m; e += blockDim.x) d[e] = sqrt(fmax(A[e * m + e].x, 0.0));
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int a = e / m, b = e % m;
        const double s = d[a] * d[b];
        Acopy[e] = s > 0.0 ? cscale(A[e], 1.0 / s) : make_double2(a == b ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) A[e] = Acopy[e];
    __syncthreads();
    if (!blk_cholesky(A, m)) {
        for (int e = tid; e < m * m; e += blockDim.x) {
            A[e] = Acopy[e];
            if (e / m == e % m) A[e].x += 1e-13 * m;
        }
        __syncthreads();
        blk_cholesky(A, m);
    }
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int b = e % m;
        A[e] = cscale(A[e], d[b] > 0.0 ? d[b] : 1.0);
    }
    __syncthreads();
}

// Per item: Gram of the r columns -> Rinv (r x r) with (A Rinv) orthonormal.
__global__ void __launch_bounds__(LB_THREADS)
chol_rinv_kernel(const double2 *__restrict__ Gram, int m, const int *__restrict__ items, double2 *__restrict__ Rinv) {
    __shared__ double2 A[LB_MAXM * LB_MAXM], B[LB_MAXM * LB_MAXM];
    __shared__ double d[LB_MAXM];
    const int b = items ? items[blockIdx.x] : blockIdx.x;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) A[e] = Gram[(int64_t)b * m * m + e];
    __syncthreads();
    scaled_cholesky(A, B, m, d);
    blk_triu_inverse(A, B, m);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) Rinv[(int64_t)b * m * m + e] = B[e];
}

// Rayleigh--Ritz-SVD step of one LOBPCG iteration for item b:
//   R = qr factor of CS (from its Gram), R = J Xi G^H (descending Xi),
//   G_X = G(:, 1:r); Hetmaniuk--Lehoucq: G_P = G_X with the X rows zeroed,
//   orthogonalised against G_X and orthonormalised in the m-dim coefficient
//   space.  m = 2r (first iteration, S = [X W]) or 3r (S = [X W P]).
//   with_p = 0 skips G_P (initial step: m = r, only Xi and G_X).
__global__ void __launch_bounds__(LB_THREADS)
lob_rr_kernel(const double2 *__restrict__ Gram, int m, int r, int with_p, const int *__restrict__ items,
              double *__restrict__ xi, double2 *__restrict__ GX, double2 *__restrict__ GP) {
    __shared__ double2 A[LB_MAXM * LB_MAXM], B[LB_MAXM * LB_MAXM], Vr[LB_MAXM * LB_MAXM];
    __shared__ double d[LB_MAXM], sig[LB_MAXM], red[224];
    __shared__ int perm[LB_MAXM];
    const int tid = threadIdx.x;
    const int b = items ? items[blockIdx.x] : blockIdx.x;
    const int MM = LB_MAXM * LB_MAXM;
    for (int e = tid; e < m * m; e += blockDim.x) A[e] = Gram[(int64_t)b * MM + e];
    __syncthreads();
    scaled_cholesky(A, B, m, d);
    blk_svd_jacobi(A, Vr, m, red);
    blk_colnorms(A, m, sig);
    if (tid == 0) {
        for (int q = 0; q < m; ++q) perm[q] = q;
        for (int q = 1; q < m; ++q) {  // descending
            int x = perm[q], w = q - 1;
            while (w >= 0 && sig[perm[w]] < sig[x]) { perm[w + 1] = perm[w]; --w; }
            perm[w + 1] = x;
        }
    }
    __syncthreads();
    // G_X (m x r) into B (ld r)
    for (int e = tid; e < m * r; e += blockDim.x) {
        const int i = e / r, c = e % r;
        B[i * r + c] = Vr[i * m + perm[c]];
    }
    if (tid < r) xi[(int64_t)b * LB_MAXM + tid] = sig[perm[tid]];
    __syncthreads();
    for (int e = tid; e < m * r; e += blockDim.x) GX[(int64_t)b * MM + e] = B[e];
    if (!with_p) return;
    // Hetmaniuk--Lehoucq: Ghat = G_X with rows 0..r-1 zeroed (A, ld r)
    for (int e = tid; e < m * r; e += blockDim.x) A[e] = (e / r) < r ? make_double2(0.0, 0.0) : B[e];
    __syncthreads();
    // Ghat -= G_X (G_X^H Ghat), twice
    for (int pass = 0; pass < 2; ++pass) {
        for (int e = tid; e < r * r; e += blockDim.x) {
            const int a = e / r, c = e % r;
            double2 s = make_double2(0.0, 0.0);
            for (int i = 0; i < m; ++i) cfma(s, cconj(B[i * r + a]), A[i * r + c]);
            Vr[e] = s;
        }
        __syncthreads();
        for (int e = tid; e < m * r; e += blockDim.x) {
            const int i = e / r, c = e % r;
            double2 s = A[e];
            for (int a = 0; a < r; ++a) cfms(s, B[i * r + a], Vr[a * r + c]);
            A[e] = s;
        }
        __syncthreads();
    }
    // orthonormalise Ghat: Gram (r x r) -> R -> Ghat R^{-1}
    double2 *Gm = Vr, *Rc = Vr + r * r, *Ri = Vr + 2 * r * r, *Cp = Vr + 3 * r * r;
    for (int e = tid; e < r * r; e += blockDim.x) {
        const int a = e / r, c = e % r;
        double2 s = make_double2(0.0, 0.0);
        for (int i = 0; i < m; ++i) cfma(s, cconj(A[i * r + a]), A[i * r + c]);
        Gm[e] = s;
    }
    __syncthreads();
    for (int e = tid; e < r * r; e += blockDim.x) Rc[e] = Gm[e];
    __syncthreads();
    scaled_cholesky(Rc, Cp, r, d);
    blk_triu_inverse(Rc, Ri, r);
    for (int e = tid; e < m * r; e += blockDim.x) {
        const int i = e / r, c = e % r;
        double2 s = make_double2(0.0, 0.0);
        for (int a = 0; a <= c; ++a) cfma(s, A[i * r + a], Ri[a * r + c]);
        GP[(int64_t)b * MM + e] = s;
    }
}

// W = Y - X diag(xi^2) for the r columns of each active item, and per item:
// ||w_1|| and the convergence decision of eq. (tolSVD) with ||C|| := xi_1
// (paper test) plus, when rtol > 0, the Kato--Temple estimate
// ||w_1||^2 / (2 xi_1^2 (xi_1^2 - xi_2^2)) <= rtol/4.
__global__ void __launch_bounds__(LB_THREADS)
lob_resid_kernel(double2 *__restrict__ S, const double2 *__restrict__ Y, int n, int64_t ld, int r,
                 const int *__restrict__ items, const double *__restrict__ xi, double eta, double rtol,
                 int *__restrict__ conv, double *__restrict__ wnorm) {
    __shared__ double red[LB_THREADS / 32][LB_MAXM / 3 + 1];
    const int tid = threadIdx.x;
    const int b = items ? items[blockIdx.x] : blockIdx.x;
    const double *xb = xi + (int64_t)b * LB_MAXM;
    double acc[LB_MAXM / 3];
#pragma unroll
    for (int c = 0; c < LB_MAXM / 3; ++c) acc[c] = 0.0;
    const int64_t x0 = (int64_t)b * 3 * r, w0 = x0 + r;
    for (int i = tid; i < n; i += blockDim.x) {
        for (int c = 0; c < r; ++c) {
            const double x2 = xb[c] * xb[c];
            const double2 yv = Y[(int64_t)i * ld + x0 + c], xv = S[(int64_t)i * ld + x0 + c];
            const double2 w = make_double2(yv.x - x2 * xv.x, yv.y - x2 * xv.y);
            S[(int64_t)i * ld + w0 + c] = w;
            acc[c] += cabs2(w);
        }
    }
    for (int c = 0; c < r; ++c) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5][c] = v;
    }
    __syncthreads();
    if (tid == 0) {
        double w1 = 0.0;
        for (int w = 0; w < LB_THREADS / 32; ++w) w1 += red[w][0];
        w1 = sqrt(w1);
        const double x1 = xb[0], x2 = r > 1 ? xb[1] : 0.0;
        bool ok = w1 <= fmax(eta * x1 * x1, x1 * x1 * 2.220446049250313e-16);
        if (ok && rtol > 0.0) {
            const double gap = x1 * x1 - x2 * x2;
            const double est = gap > 0.0 ? w1 * w1 / (2.0 * x1 * x1 * gap) : 1e300;
            ok = est <= rtol / 4.0 || w1 <= 1e-15 * x1 * x1;
        }
        conv[b] = ok ? 1 : 0;
        wnorm[b] = w1;
    }
}

// zcol[b*3r + c] = z[b] for c < 3r (shift of every column of item b)
__global__ void expand_shift_kernel(const double2 *__restrict__ z, int nitems, int r, double2 *__restrict__ zcol) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nitems * 3 * r) return;
    zcol[t] = z[t / (3 * r)];
}

// cols[t] = items[t / r] * 3r + off + t % r for t < nact * r
__global__ void make_cols_kernel(const int *__restrict__ items, int nact, int r, int off, int *__restrict__ cols) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nact * r) return;
    cols[t] = items[t / r] * 3 * r + off + t % r;
}

// dst[i][col + doff] = scale_b * src[i][col + soff] for the listed columns
// (col = the list entry, b = col / (3r)); FP64/FP32 in either direction.
template <typename S, typename D>
__global__ void copy_listed_kernel(const S *__restrict__ src, D *__restrict__ dst, int n, int64_t ld,
                                   const int *__restrict__ cols, int ncols, int soff, int doff, int r3,
                                   const double *__restrict__ scale, int sstride, int invert) {
    const int t = blockIdx.x * 32 + (threadIdx.x & 31);
    if (t >= ncols) return;
    const int col = cols[t];
    double sc = 1.0;
    if (scale) {
        const double v = scale[(int64_t)(col / r3) * sstride];
        sc = invert ? (v > 0.0 ? 1.0 / v : 1.0) : v;
    }
    for (int i = threadIdx.x >> 5; i < n; i += blockDim.x >> 5) {
        const S v = src[(int64_t)i * ld + col + soff];
        D o;
        o.x = (decltype(o.x))(sc * (double)v.x);
        o.y = (decltype(o.y))(sc * (double)v.y);
        dst[(int64_t)i * ld + col + doff] = o;
    }
}

// ------------------------------------------------------------ launchers
cudaError_t launch_chol_rinv(const double2 *Gram, int m, int nitems, const int *items, double2 *Rinv, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    note_launch(); chol_rinv_kernel<<<nitems, LB_THREADS, 0, s>>>(Gram, m, items, Rinv);
    return cudaGetLastError();
}
cudaError_t launch_lob_rr(const double2 *Gram, int m, int r, int with_p, int nitems, const int *items, double *xi,
                          double2 *GX, double2 *GP, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    note_launch(); lob_rr_kernel<<<nitems, LB_THREADS, 0, s>>>(Gram, m, r, with_p, items, xi, GX, GP);
    return cudaGetLastError();
}
cudaError_t launch_lob_resid(double2 *S, const double2 *Y, int n, int64_t ld, int r, int nitems, const int *items,
                             const double *xi, double eta, double rtol, int *conv, double *wnorm, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    note_launch(); lob_resid_kernel<<<nitems, LB_THREADS, 0, s>>>(S, Y, n, ld, r, items, xi, eta, rtol, conv, wnorm);
    return cudaGetLastError();
}
void launch_expand_shift(const double2 *z, int nitems, int r, double2 *zcol, cudaStream_t s) {
    const int t = nitems * 3 * r;
    if (t > 0) { note_launch(); expand_shift_kernel<<<(t + 255) / 256, 256, 0, s>>>(z, nitems, r, zcol); }
}
void launch_make_cols(const int *items, int nact, int r, int off, int *cols, cudaStream_t s) {
    const int t = nact * r;
    if (t > 0) { note_launch(); make_cols_kernel<<<(t + 255) / 256, 256, 0, s>>>(items, nact, r, off, cols); }
}
template <typename S, typename D>
void launch_copy_listed(const S *src, D *dst, int n, int64_t ld, const int *cols, int ncols, int soff, int doff, int r3,
                        const double *scale, int sstride, int invert, cudaStream_t s) {
    if (ncols > 0)
        note_launch(); copy_listed_kernel<S, D><<<(ncols + 31) / 32, 256, 0, s>>>(src, dst, n, ld, cols, ncols, soff, doff, r3, scale,
                                                                   sstride, invert);
}
template void launch_copy_listed<double2, double2>(const double2 *, double2 *, int, int64_t, const int *, int, int, int,
                                                   int, const double *, int, int, cudaStream_t);
template void launch_copy_listed<double2, float2>(const double2 *, float2 *, int, int64_t, const int *, int, int, int,
                                                  int, const double *, int, int, cudaStream_t);
template void launch_copy_listed<float2, double2>(const float2 *, double2 *, int, int64_t, const int *, int, int, int,
                                                  int, const double *, int, int, cudaStream_t);

}  // namespace pseudo
