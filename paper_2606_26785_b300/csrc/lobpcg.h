// Declarations of the LOBPCG-SVD kernels (lobpcg.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pseudo {
constexpr int LB_MAXM = 24;  // 3r for r <= 8
cudaError_t launch_chol_rinv(const double2 *Gram, int m, int nitems, const int *items, double2 *Rinv, cudaStream_t s);
cudaError_t launch_lob_rr(const double2 *Gram, int m, int r, int with_p, int nitems, const int *items, double *xi,
                          double2 *GX, double2 *GP, cudaStream_t s);
cudaError_t launch_lob_resid(double2 *S, const double2 *Y, int n, int64_t ld, int r, int nitems, const int *items,
                             const double *xi, double eta, double rtol, int *conv, double *wnorm, cudaStream_t s);
void launch_expand_shift(const double2 *z, int nitems, int r, double2 *zcol, cudaStream_t s);
void launch_make_cols(const int *items, int nact, int r, int off, int *cols, cudaStream_t s);
template <typename S, typename D>
void launch_copy_listed(const S *src, D *dst, int n, int64_t ld, const int *cols, int ncols, int soff, int doff, int r3,
                        const double *scale, int sstride, int invert, cudaStream_t s);
}  // namespace pseudo
