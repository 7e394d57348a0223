// Iterative refinement of shifted triangular solves in mixed precision: the
// solve runs on the FP32 panels, the residual b - (T - zI)^{op} x on the FP32
// units in double-single arithmetic, and the correction is accumulated in
// FP64.  The number of solves a column gets follows from its estimated
// condition: the error contracts by about rho = c * kappa * u_32 per step with
// kappa = (||T||_2 + |z|) / sigma, so a column gets the fewest k with rho^k
// below its accuracy target (at least 2, at most max_ir).  Columns are kept sorted by k,
// so the columns still refining at step `it` are a prefix of one list and
// every launch covers exactly them.  The plan is made on the host from host
// estimates (ir_plan) or on the device from the finished Lanczos values
// (ir_plan_dev), whose refinement launches then read their column counts from
// device memory, so that no host round trip sits between Lanczos and
// refinement.
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

// Solves a column gets: the refined vector feeds a Rayleigh quotient whose
// error is quadratic in the vector error, so a relative solve error d costs
// about (d / sigma)^2 relative in sigma and d = 1e-5 sigma / ||M(z)|| keeps
// sigma well inside 1e-8; each solve contracts the error by
// rho = 8 kappa u_32, kappa = ||M(z)|| / sigma, mz = ||T||_2 + |z|.
__host__ __device__ inline int ir_steps(double sig, double mz, double u32, int max_ir) {
    const double sg = fmax(sig, 1e-300);
    const double rho = fmin(0.5, 8.0 * (mz / sg) * u32);
    const double target = fmax(1e-15, fmin(1e-8, 1e-5 * sg / mz));
    const int k = (int)ceil(log(target) / log(rho));
    const int kc = k < max_ir ? k : max_ir;
    return kc > 2 ? kc : 2;
}

void ir_plan(pseudo_ctx *h, const std::vector<double> &sig, const std::vector<double2> &z, int max_ir,
             const IRBufs &b, IRPlan &plan, cudaStream_t s, int S_total, const std::vector<char> *skip) {
    const int S = (int)sig.size();
    if (S_total < S) S_total = S;
    std::vector<int> need(S_total, 0), perm(S);
    const double u32 = solve32_unit_roundoff(h);
    for (int c = 0; c < S; ++c) {
        const double mz = h->norm2 + std::hypot(z[c].x, z[c].y);
        need[c] = ir_steps(sig[c], mz, u32, max_ir);
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

// The device plan of the P = *nfin finished columns (one block of 1024
// threads): sigma_c = theta_c^{-1/2} from the Lanczos value; a column is
// skipped (need 0) when its recurrence did not converge, sigma_c is not
// positive, or kappa_c * u_32 > fb_ku (the FP64 pass redoes such points
// whatever the refinement gives).  perm lists the columns with need >= 1 by
// need descending, ties in column order (a stable counting sort: warp w owns
// columns [w F / 32, (w + 1) F / 32)); cnt[it] = columns with need > it for
// it = 0 .. max_ir.  stat[0] += the solves the plan makes (two directions),
// stat[1] += its residual products.
__global__ void __launch_bounds__(1024) ir_plan_kernel(const int *__restrict__ nfin, int F,
                                                       const double *__restrict__ theta, const double2 *__restrict__ z,
                                                       const int *__restrict__ conv, double norm2, double u32,
                                                       int max_ir, double fb_ku, int *__restrict__ need,
                                                       int *__restrict__ perm, int *__restrict__ cnt,
                                                       long long *__restrict__ stat) {
    __shared__ int wc[33][32];  // [need][warp] counts, then exclusive offsets
    __shared__ int tot[33], start[34];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int P = min(*nfin, F);
    const int per = (F + 31) / 32, c0 = warp * per, c1 = min(F, c0 + per);
    for (int v = lane; v <= max_ir; v += 32) wc[v][warp] = 0;
    __syncwarp();
    for (int b = c0; b < c1; b += 32) {
        const int c = b + lane;
        int v = -1;
        if (c < c1) {
            v = 0;
            if (c < P) {
                const double th = theta[c];
                const double sg = th > 0.0 ? 1.0 / sqrt(th) : 0.0;
                const double mz = norm2 + sqrt(z[c].x * z[c].x + z[c].y * z[c].y);
                const bool skip = !conv[c] || !(sg > 0.0) || (mz / sg) * u32 > fb_ku;
                v = skip ? 0 : min(ir_steps(sg, mz, u32, max_ir), max_ir);
            }
            need[c] = v;
        }
        for (int q = 1; q <= max_ir; ++q) {
            const unsigned m = __ballot_sync(0xffffffffu, v == q);
            if (lane == 0) wc[q][warp] += __popc(m);
        }
        __syncwarp();
    }
    __syncthreads();
    // per need value: exclusive scan over the warps (warp q scans need q)
    if (warp >= 1 && warp <= max_ir) {
        const int x = wc[warp][lane];
        int inc = x;
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += y;
        }
        wc[warp][lane] = inc - x;
        if (lane == 31) tot[warp] = inc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        start[max_ir + 1] = 0;
        int acc = 0;
        for (int q = max_ir; q >= 1; --q) { start[q] = acc; acc += tot[q]; }
        // columns with need > it: every need q > it
        long long solves = 0, prods = 0;
        for (int it = 0; it <= max_ir; ++it) {
            int k = 0;
            for (int q = it + 1; q <= max_ir; ++q) k += tot[q];
            cnt[it] = k;
            if (it < max_ir) solves += k;
            if (it >= 1 && it < max_ir) prods += k;
        }
        stat[0] += 2 * solves;
        stat[1] += 2 * prods;
    }
    __syncthreads();
    for (int b = c0; b < c1; b += 32) {
        const int c = b + lane;
        const int v = c < c1 ? need[c] : -1;
        for (int q = 1; q <= max_ir; ++q) {
            const unsigned m = __ballot_sync(0xffffffffu, v == q);
            if (v == q) perm[start[q] + wc[q][warp] + __popc(m & ((1u << lane) - 1u))] = c;
            __syncwarp();
            if (lane == 0) wc[q][warp] += __popc(m);
            __syncwarp();
        }
    }
}

void ir_plan_dev(pseudo_ctx *h, const int *nfin, int F, const double *theta, const double2 *z, const int *conv,
                 int max_ir, double fb_ku, const IRBufs &b, int *cnt, long long *stat, cudaStream_t s) {
    note_launch();
    ir_plan_kernel<<<1, 1024, 0, s>>>(nfin, F, theta, z, conv, h->norm2, solve32_unit_roundoff(h), max_ir, fb_ku,
                                      b.need, b.perm, cnt, stat);
}

cudaError_t ir_solve_cols_dev(pseudo_ctx *h, const IRBufs &b, int lower, const double2 *zc, int S, const double2 *B,
                              double2 *X, int max_ir, const int *cnt, cudaStream_t s) {
    const int n = h->n;
    cudaMemsetAsync(X, 0, (size_t)n * S * sizeof(double2), s);
    cudaMemcpyAsync(b.R64, B, (size_t)n * S * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < max_ir; ++it) {
        note_launch();
        need_mask_kernel<<<(S + 255) / 256, 256, 0, s>>>(b.need, it, S, b.mask);
        launch_colnorm2(b.R64, n, S, b.mask, b.rn2, s);
        launch_scale_to32(b.R64, n, S, b.mask, b.rn2, b.D32, s);
        int k0 = kp_begin(h, s);
        e = solve32(h, lower, b.perm, zc, S, cnt + it, b.D32, S, b.xs, s);
        kp_end(h, k0, PSEUDO_K_TRSV32, 0.0, 0.0, s);
        if (e != cudaSuccess) return e;
        launch_acc_from32(X, n, S, b.mask, b.rn2, b.D32, s);
        if (it + 1 < max_ir) {
            k0 = kp_begin(h, s);
            e = trmv_hp(h, true, lower, b.perm, zc, S, X, S, B, S, b.R64, S, 1, s, b.xh, b.xl, b.oz, cnt + it + 1);
            kp_end(h, k0, PSEUDO_K_TRMV_DS, 0.0, 0.0, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
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
