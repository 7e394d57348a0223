// Host side of the C ABI declared in include/pseudo.h: handle set-up (packed
// panels of T, norms), argument checking, workspace carving, and the grid
// drivers (inverse Lanczos here; recycling in recycle_driver.cu).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "pseudo.h"
#include "driver.h"

#include <atomic>

namespace pseudo {

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;
void note_launch() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++t_launches;
}
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long thread_launch_count() { return t_launches; }

static thread_local std::string g_err;

int set_err(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}
void clear_err() { g_err.clear(); }

int cuda_err(cudaError_t e, const char *where) {
    return set_err(PSEUDO_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Device arrays are read with their natural vector widths (complex values as
// 16-byte pairs, bulk copies of workspace images from 16-byte boundaries), so
// a misaligned pointer would fault on the device: it is refused on the host.
bool misaligned(const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) != 0; }

// ---------------------------------------------------------- workspace
void *Carver::take(size_t bytes) {
    size_t off = (used + 255) & ~(size_t)255;
    used = off + bytes;
    if (!base || used > cap) { overflow = true; return nullptr; }
    return base + off;
}

}  // namespace pseudo

using namespace pseudo;

extern "C" {

const char *pseudo_last_error(void) { return g_err.c_str(); }

int64_t pseudo_launch_count(void) { return (int64_t)g_launches.load(); }

int pseudo_opts_default(pseudo_opts *o) {
    if (!o) return set_err(PSEUDO_ERR_ARG, "opts is NULL");
    memset(o, 0, sizeof *o);
    o->mode = PSEUDO_INVLANC;
    o->precision = PSEUDO_FP64;
    o->r = 6;
    o->p_max = 60;
    o->batch_b = 20;
    o->eps_shift_rel = 1e-14;
    o->tau = 1e-10;
    o->omega = 1.6;
    o->eta = 1e-4;
    o->rtol = 1e-10;
    o->maxiter_lanczos = 64;
    o->maxiter_lobpcg = 60;
    o->max_ir = 6;
    o->seed = 12345;
    o->fp32_solver = PSEUDO_SOLVER_AUTO;
    o->device_loop = 1;
    return PSEUDO_OK;
}

int pseudo_create(const pseudo_c64 *T, int64_t ldT, int64_t m, int64_t n, int t_on_host, void *stream,
                  pseudo_handle *out) {
    clear_err();
    if (!out) return set_err(PSEUDO_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!T) return set_err(PSEUDO_ERR_ARG, "T is NULL");
    if (n < 1 || n > (1 << 20)) return set_err(PSEUDO_ERR_ARG, "n=%lld out of range", (long long)n);
    if (m != n && m != 2 * n)
        return set_err(PSEUDO_ERR_UNSUPPORTED, "m=%lld rows: the input is T (m = n) or the pencil [T; B] (m = 2n = %lld)",
                       (long long)m, 2 * (long long)n);
    if (ldT < m) return set_err(PSEUDO_ERR_ARG, "ldT=%lld < m=%lld", (long long)ldT, (long long)m);
    if (m == 2 * n && n > rect_max_order())
        return set_err(PSEUDO_ERR_UNSUPPORTED, "a rectangular pencil needs n <= %d", rect_max_order());
    cudaStream_t s = (cudaStream_t)stream;
    NvtxRange nr("pseudo_create: packed copies of T, norms");
    pseudo_ctx *h = new pseudo_ctx();
    h->n = (int)n;
    h->rect = m == 2 * n;
    h->n_pad = (int)((n + TC_MB - 1) / TC_MB * TC_MB);  // a multiple of both panel heights
    cudaGetDevice(&h->dev);
    const int64_t psz = packed_size(h->n_pad);
    cudaError_t e;
    double2 *Td = nullptr;
    float2 *b32 = nullptr;
    int *bad = nullptr;
    double *dsum = nullptr;
    auto fail = [&](int code) {
        if (Td && t_on_host) cudaFree(Td);
        if (b32) cudaFree(b32);
        if (bad) cudaFree(bad);
        if (dsum) cudaFree(dsum);
        pseudo_destroy(h);
        return code;
    };
    if ((e = cudaMalloc(&h->U64, psz * sizeof(double2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc U64"));
    if ((e = cudaMalloc(&h->L64, psz * sizeof(double2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc L64"));
    if ((e = cudaMalloc(&h->U32, psz * sizeof(float2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc U32"));
    if ((e = cudaMalloc(&h->L32, psz * sizeof(float2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc L32"));
    if ((e = cudaMalloc(&h->U32lo, psz * sizeof(float2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc U32lo"));
    if ((e = cudaMalloc(&h->L32lo, psz * sizeof(float2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc L32lo"));
    if ((e = cudaMalloc(&h->diag, n * sizeof(double2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc diag"));
    if ((e = cudaMalloc(&h->tcA_U, tc_pack_floats(h->n_pad) * sizeof(float) + 16)) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc tcA_U"));
    if ((e = cudaMalloc(&h->tcA_L, tc_pack_floats(h->n_pad) * sizeof(float) + 16)) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc tcA_L"));
    if ((e = cudaMalloc(&h->tcD_U, tc_diag_elems(h->n_pad) * sizeof(float2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc tcD_U"));
    if ((e = cudaMalloc(&h->tcD_L, tc_diag_elems(h->n_pad) * sizeof(float2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc tcD_L"));
    if ((e = cudaMalloc(&h->dev_err, 2 * sizeof(int))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc dev_err"));
    if ((e = cudaMalloc(&h->ozA_U, oz_a_elems(h->n_pad) * 2 + 256)) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc ozA_U"));
    if ((e = cudaMalloc(&h->ozA_L, oz_a_elems(h->n_pad) * 2 + 256)) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc ozA_L"));
    if ((e = cudaMalloc(&h->ozE_U, h->n_pad * sizeof(int))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc ozE_U"));
    if ((e = cudaMalloc(&h->ozE_L, h->n_pad * sizeof(int))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc ozE_L"));
    if ((e = cudaMemsetAsync(h->dev_err, 0, 2 * sizeof(int), s)) != cudaSuccess) return fail(cuda_err(e, "memset"));
    if ((e = cudaMalloc(&bad, 64)) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc"));
    if ((e = cudaMalloc(&dsum, 64)) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc"));
    if (t_on_host) {
        if ((e = cudaMalloc(&Td, (size_t)ldT * n * sizeof(double2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc T"));
        if ((e = cudaMemcpyAsync(Td, T, (size_t)ldT * n * sizeof(double2), cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return fail(cuda_err(e, "copy T"));
    } else {
        Td = (double2 *)T;
    }
    launch_pack_panels(Td, ldT, (int)n, h->n_pad, h->U64, h->L64, h->U32, h->L32, s);
    if (h->rect) {
        // the bottom block B (rows n .. 2n-1): FP64 panels of B and B^H (its FP32
        // panels are not kept), and the dense pencil for the per-point QR
        if ((e = cudaMalloc(&h->BU64, psz * sizeof(double2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc BU64"));
        if ((e = cudaMalloc(&h->BL64, psz * sizeof(double2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc BL64"));
        if ((e = cudaMalloc(&b32, 2 * psz * sizeof(float2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc"));
        if ((e = cudaMalloc(&h->M64, 2 * (size_t)n * n * sizeof(double2))) != cudaSuccess)
            return fail(cuda_err(e, "cudaMalloc M64"));
        launch_pack_panels(Td + n, ldT, (int)n, h->n_pad, h->BU64, h->BL64, b32, b32 + psz, s);
        if ((e = cudaMemcpy2DAsync(h->M64, 2 * n * sizeof(double2), Td, ldT * sizeof(double2), 2 * n * sizeof(double2),
                                   n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return fail(cuda_err(e, "copy M"));
    }
    launch_pack_tc(Td, ldT, (int)n, h->n_pad, h->tcA_U, h->tcA_L, h->tcD_U, h->tcD_L, s);
    launch_pack_oz(Td, ldT, (int)n, h->n_pad, h->ozA_U, h->ozA_L, h->ozE_U, h->ozE_L, s);
    launch_pack_lo(h->U64, h->U32, h->U32lo, psz, s);
    launch_pack_lo(h->L64, h->L32, h->L32lo, psz, s);
    cudaMemsetAsync(bad, 0, sizeof(int), s);
    launch_nonfinite(h->U64, psz, bad, s);
    if (h->rect) launch_nonfinite(h->BU64, psz, bad, s);
    launch_extract_diag(h->U64, (int)n, h->n_pad, h->diag, s);
    launch_sumsq(h->U64, psz, dsum, s);
    int hbad = 0;
    double fro2 = 0.0, fro2b = 0.0;
    cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&fro2, dsum, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (h->rect) {
        launch_sumsq(h->BU64, psz, dsum + 1, s);
        cudaMemcpyAsync(&fro2b, dsum + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(cuda_err(e, "pack T"));
    if (hbad) return fail(set_err(PSEUDO_ERR_NONFINITE, "T (or B) has non-finite entries in its upper triangle"));
    h->norm_fro = sqrt(fro2 + fro2b);
    // ||M||_2 estimate (M = T, or [T; B]): power iteration on M^H M from a seeded vector
    {
        double2 *x = nullptr, *y = nullptr;
        if ((e = cudaMalloc(&x, n * sizeof(double2))) != cudaSuccess) return fail(cuda_err(e, "cudaMalloc"));
        if ((e = cudaMalloc(&y, n * sizeof(double2))) != cudaSuccess) { cudaFree(x); return fail(cuda_err(e, "cudaMalloc")); }
        launch_start_vector(x, (int)n, 99, s);
        double lam = 0.0;
        double2 *yb = nullptr;
        if (h->rect && (e = cudaMalloc(&yb, 2 * n * sizeof(double2))) != cudaSuccess) {
            cudaFree(x);
            cudaFree(y);
            return fail(cuda_err(e, "cudaMalloc"));
        }
        for (int it = 0; it < 30; ++it) {
            // rectangular: x <- T^H T x + B^H B x (the current x is kept in yb)
            if (h->rect) cudaMemcpyAsync(yb, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, s);
            launch_trmv64(h->U64, (int)n, h->n_pad, 0, nullptr, nullptr, 1, nullptr, x, 1, nullptr, 1, y, 1, 0, s);
            launch_trmv64(h->L64, (int)n, h->n_pad, 1, nullptr, nullptr, 1, nullptr, y, 1, nullptr, 1, x, 1, 0, s);
            if (h->rect) {
                launch_trmv64(h->BU64, (int)n, h->n_pad, 0, nullptr, nullptr, 1, nullptr, yb, 1, nullptr, 1, y, 1, 0, s);
                launch_trmv64(h->BL64, (int)n, h->n_pad, 1, nullptr, nullptr, 1, nullptr, y, 1, nullptr, 1, yb + n, 1, 0,
                              s);
                launch_add_cols(x, yb + n, n, s);
            }
            launch_colnorm2(x, (int)n, 1, nullptr, dsum, s);
            double nx2 = 0.0;
            cudaMemcpyAsync(&nx2, dsum, sizeof(double), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            lam = sqrt(nx2);  // ||M^H M x|| for unit x
            if (!(lam > 0.0)) break;
            launch_normalize(x, (int)n, 1, nullptr, s);
        }
        cudaFree(x);
        cudaFree(y);
        if (yb) cudaFree(yb);
        h->norm2 = lam > 0.0 ? sqrt(lam) : h->norm_fro;
        if (h->norm2 > h->norm_fro) h->norm2 = h->norm_fro;
    }
    if (t_on_host) cudaFree(Td);
    Td = nullptr;
    if (b32) cudaFree(b32);
    b32 = nullptr;
    cudaFree(bad); bad = nullptr;
    cudaFree(dsum); dsum = nullptr;
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_err(e, "create"));
    memset(&h->stats, 0, sizeof h->stats);
    *out = h;
    return PSEUDO_OK;
}

int pseudo_tuned_config(int64_t n, int *fp32_solver, int *slots) {
    clear_err();
    if (n < 1) return set_err(PSEUDO_ERR_ARG, "n must be >= 1");
    if (fp32_solver) *fp32_solver = tuned_fp32_solver((int)std::min<int64_t>(n, 1 << 30));
    if (slots) *slots = tuned_slots((int)std::min<int64_t>(n, 1 << 30));
    return PSEUDO_OK;
}

int pseudo_set_wait_limit(pseudo_handle h, uint64_t ns) {
    clear_err();
    if (!h) return set_err(PSEUDO_ERR_ARG, "handle is NULL");
    h->wait_ns = ns;
    return PSEUDO_OK;
}

void pseudo_destroy(pseudo_handle h) {
    if (!h) return;
    graph_cache_free(h);
    cudaFree(h->M64);
    cudaFree(h->BU64);
    cudaFree(h->BL64);
    cudaFree(h->U64);
    cudaFree(h->L64);
    cudaFree(h->U32);
    cudaFree(h->L32);
    cudaFree(h->U32lo);
    cudaFree(h->L32lo);
    cudaFree(h->diag);
    cudaFree(h->tcA_U);
    cudaFree(h->tcA_L);
    cudaFree(h->tcD_U);
    cudaFree(h->tcD_L);
    cudaFree(h->dev_err);
    cudaFree(h->ozA_U);
    cudaFree(h->ozA_L);
    cudaFree(h->ozE_U);
    cudaFree(h->ozE_L);
    for (cudaEvent_t e : h->evs) cudaEventDestroy(e);
    delete h;
}

int pseudo_info(pseudo_handle h, int64_t *n, double *norm_fro, double *norm2_est) {
    if (!h) return set_err(PSEUDO_ERR_ARG, "handle is NULL");
    if (n) *n = h->n;
    if (norm_fro) *norm_fro = h->norm_fro;
    if (norm2_est) *norm2_est = h->norm2;
    return PSEUDO_OK;
}

int pseudo_stats(pseudo_handle h, pseudo_stats_t *out) {
    if (!h || !out) return set_err(PSEUDO_ERR_ARG, "NULL argument");
    *out = h->stats;
    return PSEUDO_OK;
}

int pseudo_stats_reset(pseudo_handle h) {
    if (!h) return set_err(PSEUDO_ERR_ARG, "handle is NULL");
    memset(&h->stats, 0, sizeof h->stats);
    memset(h->kst, 0, sizeof h->kst);
    return PSEUDO_OK;
}

int pseudo_kernel_stats(pseudo_handle h, int kclass, pseudo_kstat *out) {
    if (!h || !out || kclass < 0 || kclass >= PSEUDO_K_COUNT) return set_err(PSEUDO_ERR_ARG, "bad argument");
    *out = h->kst[kclass];
    return PSEUDO_OK;
}

// A bounded wait inside a tensor-core kernel that gave up leaves a mark in
// dev_err (the kernel returned early and its results are invalid).
static int check_dev_err(pseudo_ctx *h, cudaStream_t s) {
    int v = 0;
    cudaMemcpyAsync(&v, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e, "stream");
    if (v) {
        cudaMemsetAsync(h->dev_err, 0, sizeof(int), s);
        return set_err(PSEUDO_ERR_TIMEOUT, "a tensor-core solve timed out waiting on its pipeline");
    }
    return PSEUDO_OK;
}

int pseudo_solve_workspace_bytes(pseudo_handle h, int64_t ncols, size_t *bytes) {
    clear_err();
    if (!h || !bytes || ncols < 0 || ncols > (1 << 30)) return set_err(PSEUDO_ERR_ARG, "bad argument");
    Carver c;
    c.take(trsv_scratch_bytes(1, h->n_pad, ncols));
    c.take((size_t)h->n * ncols * sizeof(float2));
    c.take(trsv_scratch_bytes(0, h->n_pad, ncols));
    *bytes = c.used + 256;
    return PSEUDO_OK;
}

int pseudo_solve(pseudo_handle h, pseudo_c64 *X, const pseudo_c64 *z, int64_t ncols, int adjoint, int precision,
                 void *workspace, size_t workspace_bytes, void *stream) {
    clear_err();
    if (misaligned(X, 16) || misaligned(z, 16))
        return set_err(PSEUDO_ERR_ARG, "X and z must be 16-byte aligned (complex doubles)");
    if (!h || !X || !z || ncols < 0 || ncols > (1 << 30)) return set_err(PSEUDO_ERR_ARG, "bad argument");
    if (h->rect) return set_err(PSEUDO_ERR_UNSUPPORTED, "shifted solves need a square handle (m = n)");
    if (precision != PSEUDO_FP64 && precision != PSEUDO_MIXED && precision != PSEUDO_MIXED_CUDACORE &&
        precision != PSEUDO_DOUBLE_SINGLE)
        return set_err(PSEUDO_ERR_ARG, "bad precision");
    if (ncols == 0) return PSEUDO_OK;
    size_t need = 0;
    pseudo_solve_workspace_bytes(h, ncols, &need);
    if (!workspace || workspace_bytes < need) return set_err(PSEUDO_ERR_WORKSPACE, "workspace needs %zu bytes", need);
    if (misaligned(workspace, 256)) return set_err(PSEUDO_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    Carver c((char *)workspace, workspace_bytes);
    const int lower = adjoint ? 1 : 0;
    cudaError_t e;
    if (precision == PSEUDO_FP64) {
        double2 *xs = (double2 *)c.take(trsv_scratch_bytes(0, h->n_pad, ncols));
        e = launch_trsv64(lower ? h->L64 : h->U64, h->n, h->n_pad, lower, nullptr, (const double2 *)z, (int)ncols,
                          nullptr, (double2 *)X, ncols, xs, s);
    } else if (precision == PSEUDO_DOUBLE_SINGLE) {
        void *xs = c.take(trsv_ds_scratch_bytes(h->n_pad, ncols));
        e = launch_trsv_ds(h, lower, nullptr, (const double2 *)z, (int)ncols, nullptr, (double2 *)X, ncols, xs, s);
    } else {
        float2 *xs = (float2 *)c.take(trsv_scratch_bytes(1, h->n_pad, ncols));
        float2 *X32 = (float2 *)c.take((size_t)h->n * ncols * sizeof(float2));
        launch_convert_64_to_32((const double2 *)X, X32, (int64_t)h->n * ncols, s);
        const int keep = h->fp32_solver;
        h->fp32_solver = precision == PSEUDO_MIXED ? 0 : 1;
        e = solve32(h, lower, nullptr, (const double2 *)z, (int)ncols, nullptr, X32, ncols, xs, s);
        h->fp32_solver = keep;
        launch_convert_32_to_64(X32, (double2 *)X, (int64_t)h->n * ncols, s);
    }
    if (e != cudaSuccess) return cuda_err(e, "pseudo_solve");
    if (precision == PSEUDO_MIXED) {
        const int rc = check_dev_err(h, s);
        if (rc) return rc;
    }
    h->stats.sv_R += ncols;
    return PSEUDO_OK;
}

int pseudo_matvec_workspace_bytes(pseudo_handle h, int64_t ncols, size_t *bytes) {
    clear_err();
    if (!h || !bytes || ncols < 0 || ncols > (1 << 18)) return set_err(PSEUDO_ERR_ARG, "bad argument");
    *bytes = oz_scratch_bytes(h->n_pad, ncols) + 256;
    return PSEUDO_OK;
}

int pseudo_matvec(pseudo_handle h, const pseudo_c64 *X, const pseudo_c64 *B, pseudo_c64 *Y, const pseudo_c64 *z,
                  int64_t ncols, int adjoint, int subtract, int precision, void *workspace, size_t workspace_bytes,
                  void *stream) {
    clear_err();
    if (misaligned(X, 16) || misaligned(Y, 16) || misaligned(B, 16) || misaligned(z, 16))
        return set_err(PSEUDO_ERR_ARG, "X, B, Y and z must be 16-byte aligned (complex doubles)");
    if (!h || !X || !Y || ncols < 0 || (subtract && !B)) return set_err(PSEUDO_ERR_ARG, "bad argument");
    if (h->rect) return set_err(PSEUDO_ERR_UNSUPPORTED, "products with T - zI need a square handle (m = n)");
    if (precision != PSEUDO_FP64 && precision != PSEUDO_MIXED && precision != PSEUDO_MIXED_CUDACORE)
        return set_err(PSEUDO_ERR_ARG, "bad precision");
    if (ncols > (1 << 18)) return set_err(PSEUDO_ERR_ARG, "ncols too large");
    if ((const void *)X == (const void *)Y) return set_err(PSEUDO_ERR_ARG, "Y must not alias X");
    if (ncols == 0) return PSEUDO_OK;
    if (precision == PSEUDO_MIXED) {
        size_t need = 0;
        pseudo_matvec_workspace_bytes(h, ncols, &need);
        if (!workspace || workspace_bytes < need) return set_err(PSEUDO_ERR_WORKSPACE, "workspace needs %zu bytes", need);
        if (misaligned(workspace, 256)) return set_err(PSEUDO_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    }
    const int lower = adjoint ? 1 : 0;
    cudaStream_t s = (cudaStream_t)stream;
    const cudaError_t e = trmv_hp(h, precision != PSEUDO_FP64, lower, nullptr, (const double2 *)z, (int)ncols,
                                  (const double2 *)X, ncols, (const double2 *)B, ncols, (double2 *)Y, ncols, subtract,
                                  s, nullptr, nullptr, precision == PSEUDO_MIXED ? workspace : nullptr);
    if (e != cudaSuccess) return cuda_err(e, "pseudo_matvec");
    h->stats.mv_M += ncols;
    if (precision == PSEUDO_MIXED) {
        const int rc = check_dev_err(h, s);
        if (rc) return rc;
    }
    return PSEUDO_OK;
}

static int check_opts(const pseudo_opts *o) {
    if (!o) return set_err(PSEUDO_ERR_ARG, "opts is NULL");
    if (o->mode != PSEUDO_INVLANC && o->mode != PSEUDO_RECYCLE) return set_err(PSEUDO_ERR_ARG, "bad mode %d", o->mode);
    if (o->precision != PSEUDO_FP64 && o->precision != PSEUDO_MIXED) return set_err(PSEUDO_ERR_ARG, "bad precision");
    if (o->maxiter_lanczos < 1 || o->maxiter_lanczos > LANCZOS_MMAX)
        return set_err(PSEUDO_ERR_ARG, "maxiter_lanczos must be in [1, %d]", LANCZOS_MMAX);
    if (o->max_ir < 1 || o->max_ir > 32) return set_err(PSEUDO_ERR_ARG, "max_ir must be in [1, 32]");
    if (o->shift_batch < 0) return set_err(PSEUDO_ERR_ARG, "shift_batch < 0");
    if (o->fp32_solver < 0 || o->fp32_solver > PSEUDO_SOLVER_TC32) return set_err(PSEUDO_ERR_ARG, "bad fp32_solver");
    if (o->device_loop != 0 && o->device_loop != 1) return set_err(PSEUDO_ERR_ARG, "device_loop must be 0 or 1");
    if (!(o->rtol >= 0.0)) return set_err(PSEUDO_ERR_ARG, "rtol < 0");
    if (o->mode == PSEUDO_RECYCLE) {
        if (o->r < 1 || o->r > 8) return set_err(PSEUDO_ERR_ARG, "r must be in [1, 8]");
        if (o->p_max < 1) return set_err(PSEUDO_ERR_ARG, "p_max must be >= 1");
        if (!(o->omega >= 1.0)) return set_err(PSEUDO_ERR_ARG, "omega must be >= 1");
        if (o->batch_b < 1) return set_err(PSEUDO_ERR_ARG, "batch_b must be >= 1");
        if (o->grid_nx < 0 || o->grid_ny < 0) return set_err(PSEUDO_ERR_ARG, "bad grid dims");
        if (o->traversal < PSEUDO_TRAVERSE_BATCH_ZIGZAG || o->traversal > PSEUDO_TRAVERSE_MORTON)
            return set_err(PSEUDO_ERR_ARG, "bad traversal %d", o->traversal);
    }
    return PSEUDO_OK;
}

// The rectangular pencil (m = 2n) runs FP64 inverse Lanczos only.
static int check_rect(const pseudo_ctx *h, const pseudo_opts *o) {
    if (h->rect && (o->mode != PSEUDO_INVLANC || o->precision != PSEUDO_FP64))
        return set_err(PSEUDO_ERR_UNSUPPORTED, "a rectangular pencil (m = 2n) runs mode INVLANC in precision FP64 only");
    return PSEUDO_OK;
}

int pseudo_workspace_bytes(pseudo_handle h, const pseudo_opts *o, int64_t npts, size_t *bytes) {
    clear_err();
    if (!h || !bytes || npts < 0) return set_err(PSEUDO_ERR_ARG, "bad argument");
    int rc = check_opts(o);
    if (!rc) rc = check_rect(h, o);
    if (rc) return rc;
    Carver c;
    if (o->mode == PSEUDO_INVLANC) invlanc_carve(h, o, npts, c, nullptr);
    else recycle_carve(h, o, npts, c, nullptr);
    *bytes = c.used + 256;
    return PSEUDO_OK;
}

int pseudo_recycle_state_layout(pseudo_handle h, const pseudo_opts *o, int64_t npts, int64_t *out) {
    clear_err();
    if (!h || !o || !out || npts < 0) return set_err(PSEUDO_ERR_ARG, "bad argument");
    if (o->mode != PSEUDO_RECYCLE) return set_err(PSEUDO_ERR_ARG, "recycle mode only");
    int rc = check_opts(o);
    if (!rc) rc = check_rect(h, o);
    if (rc) return rc;
    recycle_state_layout(h, o, npts, out);
    return PSEUDO_OK;
}

int pseudo_grid(pseudo_handle h, const pseudo_c64 *z, int64_t npts, const double *eps_levels, int neps,
                const pseudo_opts *o, double *sigma_out, double *res_out, int32_t *flags_out, uint32_t *member_out,
                void *workspace, size_t workspace_bytes, void *stream) {
    clear_err();
    int rc = check_opts(o);
    if (rc) return rc;
    if (!o->io_host && (misaligned(z, 16) || misaligned(sigma_out, 8) || misaligned(res_out, 8) ||
                        misaligned(flags_out, 4) || misaligned(member_out, 4)))
        return set_err(PSEUDO_ERR_ARG, "device arrays must be naturally aligned (z 16, sigma/res 8, flags/member 4 "
                                       "bytes)");
    if (!h) return set_err(PSEUDO_ERR_ARG, "handle is NULL");
    rc = check_rect(h, o);
    if (rc) return rc;
    if (npts < 0 || npts >= (int64_t)1 << 31) return set_err(PSEUDO_ERR_ARG, "npts out of range");
    if (npts == 0) return PSEUDO_OK;
    if (!z || !sigma_out) return set_err(PSEUDO_ERR_ARG, "z and sigma_out are required");
    if (neps < 0 || neps > 32 || (neps > 0 && !eps_levels)) return set_err(PSEUDO_ERR_ARG, "bad eps levels");
    if (o->mode == PSEUDO_RECYCLE && o->grid_nx > 0 && (int64_t)o->grid_nx * o->grid_ny != npts)
        return set_err(PSEUDO_ERR_ARG, "grid_nx * grid_ny != npts");
    if (o->io_host) {
        for (int64_t i = 0; i < npts; ++i)
            if (!std::isfinite(z[i].re) || !std::isfinite(z[i].im)) return set_err(PSEUDO_ERR_NONFINITE, "z[%lld] is not finite", (long long)i);
    }
    size_t need = 0;
    pseudo_workspace_bytes(h, o, npts, &need);
    if (!workspace || workspace_bytes < need)
        return set_err(PSEUDO_ERR_WORKSPACE, "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes, need);
    if (((uintptr_t)workspace) & 255) return set_err(PSEUDO_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    if (!o->io_host) {
        // device shifts: one pass over z before any other work
        cudaStream_t s0 = (cudaStream_t)stream;
        int zbad = 0;
        cudaMemsetAsync(h->dev_err + 1, 0, sizeof(int), s0);
        launch_nonfinite((const double2 *)z, npts, h->dev_err + 1, s0);
        cudaMemcpyAsync(&zbad, h->dev_err + 1, sizeof(int), cudaMemcpyDeviceToHost, s0);
        const cudaError_t ez = cudaStreamSynchronize(s0);
        if (ez != cudaSuccess) return cuda_err(ez, "checking z");
        if (zbad) return set_err(PSEUDO_ERR_NONFINITE, "z has non-finite entries");
    }
    GridIO io;
    io.z = (const double2 *)z;
    io.npts = npts;
    io.eps_host = eps_levels;
    io.neps = neps;
    io.sigma = sigma_out;
    io.res = res_out;
    io.flags = flags_out;
    io.member = member_out;
    io.on_host = o->io_host != 0;
    Carver c((char *)workspace, workspace_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    h->prof = o->profile != 0;
    h->recs.clear();
    h->evn = 0;
    h->fp32_solver = o->fp32_solver == PSEUDO_SOLVER_AUTO ? tuned_fp32_solver(h->n) : o->fp32_solver;
    int res = o->mode == PSEUDO_INVLANC ? invlanc_run(h, o, io, c, s) : recycle_run(h, o, io, c, s);
    if (res >= 0 && o->precision == PSEUDO_MIXED) {
        const int rc = check_dev_err(h, s);
        if (rc) res = rc;
    }
    if (h->prof) {
        cudaStreamSynchronize(s);
        kp_resolve(h);
        h->prof = false;
    }
    return res;
}

}  // extern "C"
