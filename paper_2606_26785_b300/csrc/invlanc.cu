// Grid driver for the inverse-Lanczos method (the comparator of the paper's
// experiments, Sec. 4: Lanczos on N(z)^{-1} over Schur-triangular solves).
//
// Points are processed in waves of S shifts; inside a wave every point runs
// its own Lanczos recurrence in lock-step with the others, and converged
// points drop out of the solves (active-column list).  FP64 mode runs all of
// it in double precision.  Mixed mode runs the Lanczos recurrence on FP32
// solves and then refines each point's Ritz vector by one step of inverse
// iteration whose two solves are FP32 solves corrected by FP64 residuals
// (iterative refinement); sigma is then the FP64 Rayleigh quotient
// ||(T - zI) x|| of the refined unit vector x.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "driver.h"
#include "internal.h"

namespace pseudo {

struct LancLayout {
    int S = 0, mmax = 0;
    bool fp32 = false;
    void *Q = nullptr, *W = nullptr, *xs = nullptr;
    double2 *U = nullptr, *Y = nullptr, *NX = nullptr, *X64 = nullptr, *R64 = nullptr, *B64 = nullptr;
    double *alpha = nullptr, *beta = nullptr, *svec = nullptr, *theta = nullptr, *s2 = nullptr, *rr = nullptr,
           *rn2 = nullptr, *eps = nullptr;
    int *nsteps = nullptr, *active = nullptr, *cols = nullptr, *cnt = nullptr, *nbad = nullptr;
    double2 *startv = nullptr;
    double2 *z_dev = nullptr;
    double *sig_dev = nullptr, *res_dev = nullptr;
    int32_t *flags_dev = nullptr;
    uint32_t *member_dev = nullptr;
};

static int choose_wave(pseudo_ctx *h, const pseudo_opts *o, int64_t npts, bool fp32, int mmax) {
    int64_t S = o->shift_batch > 0 ? o->shift_batch : 8192;
    S = std::min<int64_t>(S, npts);
    const double esz = fp32 ? 8.0 : 16.0;
    while (S > 32) {
        double bytes = (double)h->n * S * ((mmax + 2) * esz + (fp32 ? 6 : 3) * 16.0);
        if (bytes <= 48e9) break;
        S /= 2;
    }
    return (int)std::max<int64_t>(S, 1);
}

static void lanc_layout(pseudo_ctx *h, const pseudo_opts *o, int64_t npts, Carver &c, LancLayout &L, bool on_host) {
    L.fp32 = o->precision == PSEUDO_MIXED;
    L.mmax = o->maxiter_lanczos;
    L.S = choose_wave(h, o, npts, L.fp32, L.mmax);
    const size_t n = h->n, S = L.S, esz = L.fp32 ? sizeof(float2) : sizeof(double2);
    L.Q = c.take((size_t)(L.mmax + 1) * n * S * esz);
    L.W = c.take(n * S * esz);
    L.xs = c.take(trsv_scratch_bytes(L.fp32 ? 1 : 0, h->n_pad, S));
    L.U = c.get<double2>(n * S);
    L.Y = c.get<double2>(n * S);
    L.NX = c.get<double2>(n * S);
    if (L.fp32) {
        L.X64 = c.get<double2>(n * S);
        L.R64 = c.get<double2>(n * S);
        L.B64 = c.get<double2>(n * S);
    }
    L.alpha = c.get<double>(S * L.mmax);
    L.beta = c.get<double>(S * L.mmax);
    L.svec = c.get<double>(S * L.mmax);
    L.theta = c.get<double>(S);
    L.s2 = c.get<double>(S);
    L.rr = c.get<double>(S);
    L.rn2 = c.get<double>(S);
    L.eps = c.get<double>(32);
    L.nsteps = c.get<int>(S);
    L.active = c.get<int>(S);
    L.cols = c.get<int>(S);
    L.cnt = c.get<int>(4);
    L.nbad = c.get<int>(4);
    L.startv = c.get<double2>(n);
    if (on_host) {
        L.z_dev = c.get<double2>(npts);
        L.sig_dev = c.get<double>(npts);
        L.res_dev = c.get<double>(npts);
        L.flags_dev = c.get<int32_t>(npts);
        L.member_dev = c.get<uint32_t>(npts);
    }
}

void invlanc_carve(pseudo_ctx *h, const pseudo_opts *o, int64_t npts, Carver &c, void *) {
    LancLayout L;
    lanc_layout(h, o, npts, c, L, o->io_host != 0);
}

// X = (T - zI)^{-op} B to FP64 accuracy by FP32 solves + FP64 residuals.
static cudaError_t ir_solve(pseudo_ctx *h, const LancLayout &L, int lower, const double2 *zc, int Sw,
                            const double2 *B, double2 *X, int max_ir, cudaStream_t s) {
    const int n = h->n;
    float2 *D32 = (float2 *)L.W;
    cudaMemsetAsync(X, 0, (size_t)n * Sw * sizeof(double2), s);
    cudaMemcpyAsync(L.R64, B, (size_t)n * Sw * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    for (int it = 0; it < max_ir; ++it) {
        launch_colnorm2(L.R64, n, Sw, nullptr, L.rn2, s);
        launch_scale_to32(L.R64, n, Sw, nullptr, L.rn2, D32, s);
        int k0 = kp_begin(h, s);
        cudaError_t e = launch_trsv32(lower ? h->L32 : h->U32, n, h->n_pad, lower, nullptr, zc, Sw, nullptr, D32, Sw,
                                      (float2 *)L.xs, s);
        kp_end(h, k0, PSEUDO_K_TRSV32, tri_flops(n, Sw), tri_bytes(n, Sw, 8, 8, 2), s);
        if (e != cudaSuccess) return e;
        launch_acc_from32(X, n, Sw, nullptr, L.rn2, D32, s);
        k0 = kp_begin(h, s);
        e = trmv_hp(h, true, lower, nullptr, zc, Sw, X, Sw, B, Sw, L.R64, Sw, 1, s);
        kp_end(h, k0, PSEUDO_K_TRMV_DS, tri_flops(n, Sw), tri_bytes(n, Sw, 16, 16, 3), s);
        if (e != cudaSuccess) return e;
        h->stats.sv_R += Sw;
        h->stats.mv_M_fp64_refine += Sw;
    }
    return cudaGetLastError();
}

int invlanc_run(pseudo_ctx *h, const pseudo_opts *o, const GridIO &io, Carver &c, cudaStream_t s) {
    LancLayout L;
    lanc_layout(h, o, io.npts, c, L, io.on_host);
    if (c.overflow) return set_err(PSEUDO_ERR_WORKSPACE, "workspace too small");
    const int n = h->n;
    const int64_t npts = io.npts;
    cudaError_t e;
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, s);

    const double2 *zall = io.z;
    double *sig_all = io.sigma, *res_all = io.res;
    int32_t *flags_all = io.flags;
    uint32_t *member_all = io.member;
    if (io.on_host) {
        cudaMemcpyAsync(L.z_dev, io.z, npts * sizeof(double2), cudaMemcpyHostToDevice, s);
        zall = L.z_dev;
        sig_all = L.sig_dev;
        res_all = io.res ? L.res_dev : nullptr;
        flags_all = io.flags ? L.flags_dev : nullptr;
        member_all = io.member ? L.member_dev : nullptr;
    }
    if (io.neps > 0) cudaMemcpyAsync(L.eps, io.eps_host, io.neps * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(L.nbad, 0, sizeof(int), s);
    launch_start_vector(L.startv, n, o->seed, s);

    const double rt = o->rtol > 0.0 ? o->rtol : 1e-8;
    const double tol_q = L.fp32 ? 1e-10 : rt / 2.0;
    const double tol_floor = L.fp32 ? 1e-6 : 1e-15;

    for (int64_t w0 = 0; w0 < npts; w0 += L.S) {
        const int Sw = (int)std::min<int64_t>(L.S, npts - w0);
        const double2 *zc = zall + w0;
        const int64_t qs = (int64_t)n * Sw;
        launch_fill_int(L.active, Sw, 1, s);
        if (L.fp32) launch_bcast_start<float>(L.startv, n, Sw, (float2 *)L.Q, s);
        else launch_bcast_start<double>(L.startv, n, Sw, (double2 *)L.Q, s);
        launch_compact_active(L.active, Sw, L.cols, L.cnt, s);
        int ncnt = Sw;
        for (int j = 0; j < L.mmax && ncnt > 0; ++j) {
            if (L.fp32) {
                float2 *Q = (float2 *)L.Q, *W = (float2 *)L.W;
                launch_copy_cols<float>(Q + (int64_t)j * qs, W, n, Sw, L.active, s);
                int k0 = kp_begin(h, s);
                e = launch_trsv32(h->L32, n, h->n_pad, 1, L.cols, zc, ncnt, L.cnt, W, Sw, (float2 *)L.xs, s);
                kp_end(h, k0, PSEUDO_K_TRSV32, tri_flops(n, ncnt), tri_bytes(n, ncnt, 8, 8, 2), s);
                k0 = kp_begin(h, s);
                if (e == cudaSuccess)
                    e = launch_trsv32(h->U32, n, h->n_pad, 0, L.cols, zc, ncnt, L.cnt, W, Sw, (float2 *)L.xs, s);
                kp_end(h, k0, PSEUDO_K_TRSV32, tri_flops(n, ncnt), tri_bytes(n, ncnt, 8, 8, 2), s);
                k0 = kp_begin(h, s);
                launch_lanczos_orth<float>(Q, qs, W, n, Sw, j, L.mmax, L.active, L.alpha, L.beta, s);
                kp_end(h, k0, PSEUDO_K_LANCZOS, 32.0 * (j + 1) * n * ncnt, 4.0 * (j + 2) * n * ncnt * 8, s);
            } else {
                double2 *Q = (double2 *)L.Q, *W = (double2 *)L.W;
                launch_copy_cols<double>(Q + (int64_t)j * qs, W, n, Sw, L.active, s);
                int k0 = kp_begin(h, s);
                e = launch_trsv64(h->L64, n, h->n_pad, 1, L.cols, zc, ncnt, L.cnt, W, Sw, (double2 *)L.xs, s);
                kp_end(h, k0, PSEUDO_K_TRSV64, tri_flops(n, ncnt), tri_bytes(n, ncnt, 16, 16, 2), s);
                k0 = kp_begin(h, s);
                if (e == cudaSuccess)
                    e = launch_trsv64(h->U64, n, h->n_pad, 0, L.cols, zc, ncnt, L.cnt, W, Sw, (double2 *)L.xs, s);
                kp_end(h, k0, PSEUDO_K_TRSV64, tri_flops(n, ncnt), tri_bytes(n, ncnt, 16, 16, 2), s);
                k0 = kp_begin(h, s);
                launch_lanczos_orth<double>(Q, qs, W, n, Sw, j, L.mmax, L.active, L.alpha, L.beta, s);
                kp_end(h, k0, PSEUDO_K_LANCZOS, 32.0 * (j + 1) * n * ncnt, 4.0 * (j + 2) * n * ncnt * 16, s);
            }
            if (e != cudaSuccess) return cuda_err(e, "lanczos solve");
            h->stats.sv_R += 2 * (int64_t)ncnt;
            h->stats.lanczos_steps += 1;
            launch_lanczos_tridiag(Sw, j, L.mmax, L.alpha, L.beta, L.active, L.theta, L.svec, L.nsteps, tol_q,
                                   tol_floor, j == L.mmax - 1, s);
            launch_compact_active(L.active, Sw, L.cols, L.cnt, s);
            cudaMemcpyAsync(&ncnt, L.cnt, sizeof(int), cudaMemcpyDeviceToHost, s);
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_err(e, "lanczos step");
        }
        if (L.fp32) launch_ritz_vector<float>((const float2 *)L.Q, qs, n, Sw, L.mmax, L.svec, L.nsteps, L.U, nullptr, s);
        else launch_ritz_vector<double>((const double2 *)L.Q, qs, n, Sw, L.mmax, L.svec, L.nsteps, L.U, nullptr, s);
        if (L.fp32) {
            // one step of inverse iteration on N(z) with refined solves
            if ((e = ir_solve(h, L, 1, zc, Sw, L.U, L.X64, o->max_ir, s)) != cudaSuccess) return cuda_err(e, "refine");
            cudaMemcpyAsync(L.B64, L.X64, (size_t)n * Sw * sizeof(double2), cudaMemcpyDeviceToDevice, s);
            if ((e = ir_solve(h, L, 0, zc, Sw, L.B64, L.X64, o->max_ir, s)) != cudaSuccess) return cuda_err(e, "refine");
            launch_normalize(L.X64, n, Sw, nullptr, s);
            cudaMemcpyAsync(L.U, L.X64, (size_t)n * Sw * sizeof(double2), cudaMemcpyDeviceToDevice, s);
        }
        // Rayleigh quotient and residual of the returned vector, in FP64
        {
            const int kc = L.fp32 ? PSEUDO_K_TRMV_DS : PSEUDO_K_TRMV64;
            int k0 = kp_begin(h, s);
            trmv_hp(h, L.fp32, 0, nullptr, zc, Sw, L.U, Sw, nullptr, Sw, L.Y, Sw, 0, s);
            trmv_hp(h, L.fp32, 1, nullptr, zc, Sw, L.Y, Sw, nullptr, Sw, L.NX, Sw, 0, s);
            kp_end(h, k0, kc, 2 * tri_flops(n, Sw), 2 * tri_bytes(n, Sw, 16, 16, 2), s);
        }
        h->stats.mv_M_fp64_refine += 2 * (int64_t)Sw;
        launch_rq_residual(L.U, L.Y, L.NX, n, Sw, nullptr, L.s2, L.rr, s);
        launch_finalize(Sw, w0, zc, L.theta, L.s2, L.rr, L.active, nullptr, L.fp32 ? 1 : 0, h->norm2, L.eps, io.neps,
                        sig_all, res_all, flags_all, member_all, PSEUDO_PT_REFINED, L.nbad, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "wave");
    }
    if (io.on_host) {
        cudaMemcpyAsync(io.sigma, sig_all, npts * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (io.res) cudaMemcpyAsync(io.res, res_all, npts * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (io.flags) cudaMemcpyAsync(io.flags, flags_all, npts * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (io.member) cudaMemcpyAsync(io.member, member_all, npts * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    }
    int nbad = 0;
    cudaMemcpyAsync(&nbad, L.nbad, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaEventRecord(ev1, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_err(e, "pseudo_grid");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    h->stats.ms_total += ms;
    h->stats.n_points += npts;
    h->stats.n_refined += npts;
    h->stats.n_not_converged += nbad;
    return nbad ? PSEUDO_WARN_NOT_CONVERGED : PSEUDO_OK;
}

}  // namespace pseudo
