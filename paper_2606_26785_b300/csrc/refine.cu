// Iterative refinement of shifted triangular solves in mixed precision: the
// solve runs on the FP32 panels, the residual b - (T - zI)^{op} x on the FP32
// units in double-single arithmetic, and the correction is accumulated in
// FP64.  The number of solves a column gets follows from its estimated
// condition: the error contracts by about rho = c * kappa * u_32 per step with
// kappa = (||T||_2 + |z|) / sigma, so a column gets the fewest k with rho^k
// below its accuracy target (at least 2, at most max_ir).  Columns are kept sorted by k,
// so the columns still refining at step `it` are a prefix of one list and
// every launch covers exactly them.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "common.cuh"
#include "driver.h"
#include "internal.h"

namespace pseudo {

__global__ void need_mask_kernel(const int *__restrict__ need, int it, int S, int *__restrict__ mask) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < S) mask[c] = need[c] > it ? 1 : 0;
}

void ir_plan(pseudo_ctx *h, const std::vector<double> &sig, const std::vector<double2> &z, int max_ir,
             const IRBufs &b, IRPlan &plan, cudaStream_t s, int S_total, const std::vector<char> *skip) {
    const int S = (int)sig.size();
    if (S_total < S) S_total = S;
    std::vector<int> need(S_total, 0), perm(S);
    const double u32 = solve32_unit_roundoff(h);
    for (int c = 0; c < S; ++c) {
        // The refined vector feeds a Rayleigh quotient whose error is quadratic
        // in the vector error: a relative solve error d costs about (d / sigma)^2
        // relative in sigma, so d = 1e-5 sigma / ||M(z)|| keeps sigma well inside
        // 1e-8.
        const double mz = h->norm2 + std::hypot(z[c].x, z[c].y);
        const double sg = std::max(sig[c], 1e-300);
        const double kappa = mz / sg;
        const double rho = std::min(0.5, 8.0 * kappa * u32);
        const double target = std::max(1e-15, std::min(1e-8, 1e-5 * sg / mz));
        int k = (int)std::ceil(std::log(target) / std::log(rho));
        need[c] = std::max(2, std::min(max_ir, k));
        if (skip && (*skip)[c]) need[c] = 0;
    }
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int c) { return need[a] > need[c]; });
    const int kmax = S ? need[perm[0]] : 0;
    plan.cnt.assign(kmax + 1, 0);
    for (int c = 0; c < S; ++c)
        for (int it = 0; it < need[c]; ++it) plan.cnt[it] += 1;
    cudaMemcpyAsync(b.need, need.data(), S_total * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b.perm, perm.data(), S * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);  // the host vectors go out of scope
}

cudaError_t ir_solve_cols(pseudo_ctx *h, const IRBufs &b, int lower, const double2 *zc, int S, const double2 *B,
                          double2 *X, const IRPlan &plan, cudaStream_t s) {
    const int n = h->n;
    cudaMemsetAsync(X, 0, (size_t)n * S * sizeof(double2), s);
    cudaMemcpyAsync(b.R64, B, (size_t)n * S * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    cudaError_t e = cudaSuccess;
    for (size_t it = 0; it + 1 < plan.cnt.size() && plan.cnt[it] > 0; ++it) {
        const int cnt = plan.cnt[it], next = plan.cnt[it + 1];
        note_launch();
        need_mask_kernel<<<(S + 255) / 256, 256, 0, s>>>(b.need, (int)it, S, b.mask);
        launch_colnorm2(b.R64, n, S, b.mask, b.rn2, s);
        launch_scale_to32(b.R64, n, S, b.mask, b.rn2, b.D32, s);
        int k0 = kp_begin(h, s);
        e = solve32(h, lower, b.perm, zc, cnt, nullptr, b.D32, S, b.xs, s);
        kp_end(h, k0, PSEUDO_K_TRSV32, tri_flops(n, cnt), tri_bytes(n, cnt, 8, 8, 2), s);
        if (e != cudaSuccess) return e;
        launch_acc_from32(X, n, S, b.mask, b.rn2, b.D32, s);
        h->stats.sv_R += cnt;
        if (next > 0) {
            k0 = kp_begin(h, s);
            e = trmv_hp(h, true, lower, b.perm, zc, next, X, S, B, S, b.R64, S, 1, s, b.xh, b.xl, b.oz);
            kp_end(h, k0, PSEUDO_K_TRMV_DS, tri_flops(n, next), tri_bytes(n, next, 16, 16, 3), s);
            if (e != cudaSuccess) return e;
            h->stats.mv_M_fp64_refine += next;
        }
    }
    return cudaGetLastError();
}

}  // namespace pseudo
