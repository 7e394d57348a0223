// Batched tall-skinny kernels in FP64 for the recycled subspace and the
// LOBPCG-SVD refinement: for every batch item b (a recycle lane or a refined
// grid point) with n x ka block A_b and n x kb block B_b (row-major, leading
// dimension ld, item stride bs):
//   ts_gram : G_b = A_b^H B_b            (ka x kb, accumulated over row slices)
//   ts_mul  : O_b = beta O_b + A_b C_b   (C_b is ka x kb)
// Rows are split over CTAs (grid.y) so that even a single item fills the GPU;
// partial Grams are summed with FP64 atomics into a zeroed output.
#include "common.cuh"
#include "internal.h"

namespace pseudo {

constexpr int TS_ROWS = 128;   // rows per CTA slice in ts_gram
constexpr int TS_THREADS = 256;

__global__ void __launch_bounds__(TS_THREADS)
ts_gram_kernel(TSView A, int ka, TSView B, int kb, int n, const int *__restrict__ items, double2 *__restrict__ G,
               int64_t gstride, int slice) {
    extern __shared__ double2 sh[];  // [slice][ka] then [slice][kb]
    const int b = items ? items[blockIdx.x] : blockIdx.x;
    const int r0 = blockIdx.y * slice;
    const int rows = min(slice, n - r0);
    if (rows <= 0) return;
    double2 *sa = sh, *sb = sh + slice * ka;
    const double2 *Ab = A.at(b), *Bb = B.at(b);
    for (int e = threadIdx.x; e < rows * ka; e += blockDim.x) {
        const int i = e / ka, j = e % ka;
        sa[i * ka + j] = Ab[(int64_t)(r0 + i) * A.ld + j];
    }
    for (int e = threadIdx.x; e < rows * kb; e += blockDim.x) {
        const int i = e / kb, j = e % kb;
        sb[i * kb + j] = Bb[(int64_t)(r0 + i) * B.ld + j];
    }
    __syncthreads();
    double2 *Gb = G + (int64_t)b * gstride;
    for (int e = threadIdx.x; e < ka * kb; e += blockDim.x) {
        const int a = e / kb, c = e % kb;
        double sr = 0.0, si = 0.0;
        for (int i = 0; i < rows; ++i) {
            const double2 x = sa[i * ka + a], y = sb[i * kb + c];
            sr += x.x * y.x + x.y * y.y;
            si += x.x * y.y - x.y * y.x;
        }
        atomicAdd(&Gb[a * kb + c].x, sr);
        atomicAdd(&Gb[a * kb + c].y, si);
    }
}

// O = beta*O + alpha*(A C) ; C per item (ka x kb row-major, stride cstride).  O must
// not overlap A.
__global__ void __launch_bounds__(TS_THREADS)
ts_mul_kernel(TSView A, int ka, const double2 *__restrict__ C, int64_t cstride, TSView O, int kb, int n,
              const int *__restrict__ items, double beta, double alpha) {
    extern __shared__ double2 sc[];  // C_b
    const int b = items ? items[blockIdx.x] : blockIdx.x;
    const double2 *Cb = C + (int64_t)b * cstride;
    for (int e = threadIdx.x; e < ka * kb; e += blockDim.x) sc[e] = Cb[e];
    __syncthreads();
    const double2 *Ab = A.at(b);
    double2 *Ob = O.at(b);
    const int r0 = blockIdx.y * TS_ROWS;
    const int rows = min(TS_ROWS, n - r0);
    for (int e = threadIdx.x; e < rows * kb; e += blockDim.x) {
        const int i = r0 + e / kb, c = e % kb;
        const double2 *ar = Ab + (int64_t)i * A.ld;
        double2 acc = make_double2(0.0, 0.0);
        for (int a = 0; a < ka; ++a) cfma(acc, ar[a], sc[a * kb + c]);
        double2 *o = Ob + (int64_t)i * O.ld + c;
        acc.x *= alpha; acc.y *= alpha;
        if (beta != 0.0) { acc.x += beta * o->x; acc.y += beta * o->y; }
        *o = acc;
    }
}

cudaError_t launch_ts_gram(TSView A, int ka, TSView B, int kb, int n, int nitems, const int *items, double2 *G,
                           int64_t gstride, bool zero, cudaStream_t s) {
    if (nitems <= 0 || ka <= 0 || kb <= 0) return cudaSuccess;
    // zero: clear items 0..nitems-1 of G (only valid without an item list)
    if (zero) cudaMemsetAsync(G, 0, sizeof(double2) * (size_t)gstride * nitems, s);
    int slice = (96 * 1024) / (int)(sizeof(double2) * (ka + kb));
    slice = slice > TS_ROWS ? TS_ROWS : slice;
    if (slice < 1) slice = 1;
    size_t sm = sizeof(double2) * (size_t)slice * (ka + kb);
    static std::atomic<uint64_t> attr{0};
    smem_attr_once(ts_gram_kernel, 160 * 1024, attr);
    dim3 grid(nitems, (n + slice - 1) / slice);
    note_launch(); ts_gram_kernel<<<grid, TS_THREADS, sm, s>>>(A, ka, B, kb, n, items, G, gstride, slice);
    return cudaGetLastError();
}

cudaError_t launch_ts_mul(TSView A, int ka, const double2 *C, int64_t cstride, TSView O, int kb, int n, int nitems,
                          const int *items, double beta, double alpha, cudaStream_t s) {
    if (nitems <= 0 || kb <= 0) return cudaSuccess;
    size_t sm = sizeof(double2) * (size_t)(ka > 0 ? ka : 1) * kb;
    static std::atomic<uint64_t> attr{0};
    smem_attr_once(ts_mul_kernel, 160 * 1024, attr);
    dim3 grid(nitems, (n + TS_ROWS - 1) / TS_ROWS);
    note_launch(); ts_mul_kernel<<<grid, TS_THREADS, sm, s>>>(A, ka, C, cstride, O, kb, n, items, beta, alpha);
    return cudaGetLastError();
}

}  // namespace pseudo
