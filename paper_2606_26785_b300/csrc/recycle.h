// Declarations shared by the recycling kernels and their driver.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pseudo {

constexpr int RTMAX = 16;  // cap on r~ (columns kept in the second Rayleigh--Ritz step)

struct RecySingLaunch {
    int n, KM, r, npts;
    int64_t ldv;  // row stride of V, W1, W3, W4 (lanes interleaved by column blocks of KM)
    const double2 *V, *W1, *W3, *W4, *H1, *H2;
    const int *p;
    const double2 *z;
    const int *lane;
    double eps_shift, tau, eta, rtol, norm2;
    double *sigma, *res, *xi2, *w2;
    int *accept, *rt;
    double2 *CX;
};
size_t recysing_smem(int KM);
cudaError_t launch_recysing(const RecySingLaunch &L, cudaStream_t s);

}  // namespace pseudo
