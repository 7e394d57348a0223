// Grid driver of the recycling method (Alg. 3, psTriRecy) on the GPU.
//
// Traversal (Sec. 2.3): the grid is cut into column batches of b points and
// visited batch-row by batch-row in a zigzag, each batch bottom-up.  The
// visiting sequence is split into `lanes` contiguous segments; every lane
// keeps its own recycled subspace and walks its segment in the paper's order,
// and the lanes advance side by side in rounds.  In one round each lane
// takes its next batch (a single point while its subspace is still empty):
//   1. recySing for all points of the round against the lanes' current
//      subspaces (frozen during the round),
//   2. the rejected points are refined together by LOBPCG-SVD on
//      (T - zI)^{-H} (shift-batched multi-shift solves),
//   3. [mixed precision] the first refined singular vector of each point is
//      polished by one step of inverse iteration with FP64-corrected solves,
//   4. updateRecy is applied per lane, in the lane's visiting order.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "driver.h"
#include "internal.h"
#include "lobpcg.h"
#include "recycle.h"

namespace pseudo {

// ---------------------------------------------------------------- kernels
__global__ void gather_z_kernel(const double2 *__restrict__ z, const int *__restrict__ idx, int cnt,
                                double2 *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) out[t] = z[idx[t]];
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// seeded random block (columns [j*3r, j*3r + r) of S) for the listed points
__global__ void rand_block_kernel(double2 *__restrict__ S, int n, int64_t ld, int r, const int *__restrict__ items,
                                  int nitems, const int *__restrict__ gidx, uint64_t seed) {
    const int b = blockIdx.y;
    if (b >= nitems) return;
    const int j = items[b];
    const uint64_t g = (uint64_t)gidx[j];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * r; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / r, c = e % r;
        const uint64_t key = seed * 0x100000001B3ull ^ (g * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)(i * 16 + c) << 1);
        const uint64_t a = mix64(key), bb = mix64(key + 1);
        S[i * ld + (int64_t)j * 3 * r + c] =
            make_double2((double)(a >> 11) * (1.0 / 9007199254740992.0) - 0.5, (double)(bb >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    }
}

// Write results of round points: sigma/res/flags/member at global index gidx[j]
__global__ void scatter_round_kernel(const int *__restrict__ list, int cnt, const int *__restrict__ gidx,
                                     const double *__restrict__ sig, const double *__restrict__ res, int flag,
                                     const double *__restrict__ eps, int neps, double *__restrict__ sigma_out,
                                     double *__restrict__ res_out, int32_t *__restrict__ flags_out,
                                     uint32_t *__restrict__ member_out, const int *__restrict__ nconv_flags) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int j = list ? list[t] : t;
    const int g = gidx[j];
    const double s = sig[j];
    sigma_out[g] = s;
    if (res_out) res_out[g] = res[j];
    if (flags_out) flags_out[g] = flag | (nconv_flags ? nconv_flags[j] : 0);
    if (member_out) {
        uint32_t m = 0;
        for (int e = 0; e < neps; ++e) m |= (s < eps[e] ? 1u : 0u) << e;
        member_out[g] = m;
    }
}

// Refined points: sigma from LOBPCG (1/xi_1) or from the polished Rayleigh
// quotient; res from the returned vector.
__global__ void refined_values_kernel(const int *__restrict__ items, int cnt, const double *__restrict__ xi,
                                      const double *__restrict__ s2, const double *__restrict__ rr,
                                      const double2 *__restrict__ zr, double norm2, int use_rq,
                                      double *__restrict__ sig, double *__restrict__ res) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int j = items[t];
    const double x1 = xi[(int64_t)j * LB_MAXM];
    const double rq = sqrt(fmax(s2[t], 0.0));
    const double s = use_rq ? rq : (x1 > 0.0 ? 1.0 / x1 : 0.0);
    const double2 z = zr[j];
    const double mz = norm2 + sqrt(z.x * z.x + z.y * z.y);
    sig[j] = s;
    res[j] = rq > 0.0 ? rr[t] / (rq * mz) : 0.0;
}

// U[:, t] <- S[:, items[t]*3r] (the first Ritz vector of each refined point), and back
__global__ void x1_gather_kernel(const double2 *__restrict__ S, int64_t ld, int r, const int *__restrict__ items,
                                 int cnt, int n, double2 *__restrict__ U, const double2 *__restrict__ zr,
                                 double2 *__restrict__ zc, int back) {
    const int t = blockIdx.x * 32 + (threadIdx.x & 31);
    if (t >= cnt) return;
    const int j = items[t];
    if (!back && (threadIdx.x >> 5) == 0) zc[t] = zr[j];
    for (int i = threadIdx.x >> 5; i < n; i += blockDim.x >> 5) {
        if (back) ((double2 *)S)[(int64_t)i * ld + (int64_t)j * 3 * r] = U[(int64_t)i * cnt + t];
        else U[(int64_t)i * cnt + t] = S[(int64_t)i * ld + (int64_t)j * 3 * r];
    }
}

// cols[u*r + c] = lanes[u]*KM + kk[u] + c
__global__ void lane_cols_kernel(const int *__restrict__ lanes, const int *__restrict__ kk, int nu, int r, int KM,
                                 int *__restrict__ cols) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nu * r) return;
    const int u = t / r;
    cols[t] = lanes[u] * KM + kk[u] + t % r;
}

// ---------------------------------------------------------------- layout
struct RecyLayout {
    int L = 0, KM = 0, r = 0, b = 0, B = 0, Ld = 0, Wd = 0;
    bool fp32 = false;
    double2 *V, *W1, *W3, *W4, *H1, *H2, *Lf;
    int *p;
    // round buffers (indexed by round point j < B)
    double2 *zr, *CX;
    int *lane_r, *acc_r, *rt_r, *ridx, *items, *cols, *conv, *nflag;
    double *sig_r, *res_r, *xi2_r, *w2_r, *xi, *wnorm;
    // LOBPCG
    double2 *S, *CS, *Sn, *CSn, *Yb, *zcol, *Gm, *GX, *GP, *Gr, *Rinv;
    float2 *SB32;
    void *xs;
    // polish / residual (compact, up to B columns)
    double2 *U, *Y, *NX, *X64, *R64, *B64, *zc;
    float2 *D32;
    float2 *xh, *xl;  // FP32 split of a product operand, n x max(B, lanes * k_max)
    void *oz;         // tensor-core product scratch (unused: see recycle_carve)
    int *need, *perm, *mask;  // refinement plan of the polish
    double *rn2, *s2, *rr;
    // update (slots up to L)
    double2 *Xst, *Xt2, *Cc, *C2, *gx, *Rn, *Rni, *R2, *R2i, *Rf, *Hc1, *Hc2, *Hr2, *Qacc, *Tmp;
    int *slot_lanes, *slot_items, *lout, *kk, *ucols, *nskip;
    // io
    double *eps;
    int *gidx_all, *lane_all;
    double2 *z_dev;
    double *sig_dev, *res_dev;
    int32_t *flags_dev;
    uint32_t *member_dev;
};

static int auto_lanes(const pseudo_opts *o, int64_t npts) {
    if (o->lanes > 0) return o->lanes;
    const int64_t b = std::max(1, o->batch_b);
    const int64_t nb = (npts + b - 1) / b;
    // about 50 batches per lane, between 1 and 64 lanes
    return (int)std::max<int64_t>(1, std::min<int64_t>(64, nb / 50));
}

static void recy_layout(pseudo_ctx *h, const pseudo_opts *o, int64_t npts, Carver &c, RecyLayout &R, bool on_host) {
    R.r = o->r;
    R.KM = std::min(o->p_max, RECY_KMAX / o->r) * o->r;  // p_max is capped at RECY_KMAX / r
    // points a lane takes per round: 1 keeps the paper's point-by-point
    // recycling inside every lane (V updated after each refined point)
    R.b = o->shift_batch > 0 ? o->shift_batch : 1;
    R.L = auto_lanes(o, npts);
    R.B = R.L * R.b;
    R.Ld = R.L * R.KM;
    R.Wd = R.B * 3 * R.r;
    R.fp32 = o->precision == PSEUDO_MIXED;
    const size_t n = h->n, L = R.L, KM = R.KM, r = R.r, B = R.B, Wd = R.Wd, MM = LB_MAXM * LB_MAXM;
    R.V = c.get<double2>(n * R.Ld);
    R.W1 = c.get<double2>(n * R.Ld);
    R.W3 = c.get<double2>(n * R.Ld);
    R.W4 = c.get<double2>(n * R.Ld);
    R.H1 = c.get<double2>(L * KM * KM);
    R.H2 = c.get<double2>(L * KM * KM);
    R.Lf = c.get<double2>(L * KM * KM);
    R.p = c.get<int>(L);
    R.zr = c.get<double2>(B);
    R.CX = c.get<double2>(B * KM * r);
    R.lane_r = c.get<int>(B);
    R.acc_r = c.get<int>(B);
    R.rt_r = c.get<int>(B);
    R.ridx = c.get<int>(B);
    R.items = c.get<int>(B);
    R.cols = c.get<int>(Wd);
    R.conv = c.get<int>(B);
    R.nflag = c.get<int>(B);
    R.sig_r = c.get<double>(B);
    R.res_r = c.get<double>(B);
    R.xi2_r = c.get<double>(B);
    R.w2_r = c.get<double>(B);
    R.xi = c.get<double>(B * LB_MAXM);
    R.wnorm = c.get<double>(B);
    R.S = c.get<double2>(n * Wd);
    R.CS = c.get<double2>(n * Wd);
    R.Sn = c.get<double2>(n * Wd);
    R.CSn = c.get<double2>(n * Wd);
    R.Yb = c.get<double2>(n * Wd);
    R.zcol = c.get<double2>(Wd);
    R.Gm = c.get<double2>(B * MM);
    R.GX = c.get<double2>(B * MM);
    R.GP = c.get<double2>(B * MM);
    R.Gr = c.get<double2>(B * r * r);
    R.Rinv = c.get<double2>(B * r * r);
    R.SB32 = R.fp32 ? c.get<float2>(n * Wd) : nullptr;
    R.xs = c.take(std::max(trsv_scratch_bytes(R.fp32 ? 1 : 0, h->n_pad, Wd), trsv_scratch_bytes(1, h->n_pad, B)));
    R.U = c.get<double2>(n * B);
    R.Y = c.get<double2>(n * B);
    R.NX = c.get<double2>(n * B);
    R.X64 = c.get<double2>(n * B);
    R.R64 = c.get<double2>(n * B);
    R.B64 = c.get<double2>(n * B);
    R.zc = c.get<double2>(B);
    R.D32 = c.get<float2>(n * B);
    R.xh = c.get<float2>(n * std::max<size_t>(B, R.Ld));
    R.xl = c.get<float2>(n * std::max<size_t>(B, R.Ld));
    // The recycling path keeps the CUDA-core double-single products: it has no
    // FP64 fallback, and near-singular points (sigma far below ||T|| ||x||) need
    // the element-wise accuracy of double-single, which the column-scaled
    // tensor-core slicing does not give for strongly graded vectors.
    R.oz = nullptr;
    R.need = c.get<int>(B);
    R.perm = c.get<int>(B);
    R.mask = c.get<int>(B);
    R.rn2 = c.get<double>(B);
    R.s2 = c.get<double>(B);
    R.rr = c.get<double>(B);
    R.Xst = c.get<double2>(n * L * r);
    R.Xt2 = c.get<double2>(n * L * r);
    R.Cc = c.get<double2>(L * KM * r);
    R.C2 = c.get<double2>(L * KM * r);
    R.gx = c.get<double2>(L * r * r);
    R.Rn = c.get<double2>(L * r * r);
    R.Rni = c.get<double2>(L * r * r);
    R.R2 = c.get<double2>(L * r * r);
    R.R2i = c.get<double2>(L * r * r);
    R.Rf = c.get<double2>(L * r * r);
    R.Hc1 = c.get<double2>(L * KM * r);
    R.Hc2 = c.get<double2>(L * KM * r);
    R.Hr2 = c.get<double2>(L * r * KM);
    R.Qacc = c.get<double2>(L * KM * KM);
    R.Tmp = c.get<double2>(n * L * KM);
    R.slot_lanes = c.get<int>(L);
    R.slot_items = c.get<int>(L);
    R.lout = c.get<int>(L);
    R.kk = c.get<int>(L);
    R.ucols = c.get<int>(L * r);
    R.nskip = c.get<int>(4);
    R.eps = c.get<double>(32);
    R.gidx_all = c.get<int>(npts);
    R.lane_all = c.get<int>(npts);
    if (on_host) {
        R.z_dev = c.get<double2>(npts);
        R.sig_dev = c.get<double>(npts);
        R.res_dev = c.get<double>(npts);
        R.flags_dev = c.get<int32_t>(npts);
        R.member_dev = c.get<uint32_t>(npts);
    } else {
        R.z_dev = nullptr; R.sig_dev = nullptr; R.res_dev = nullptr; R.flags_dev = nullptr; R.member_dev = nullptr;
    }
}

void recycle_carve(pseudo_ctx *h, const pseudo_opts *o, int64_t npts, Carver &c, void *) {
    RecyLayout R;
    recy_layout(h, o, npts, c, R, o->io_host != 0);
}

// Where the lanes' recycle state sits in the workspace after pseudo_grid:
// out = {lanes, k_max, row stride of V/W (elements), byte offsets of V, W1,
// W3, W4, H1, H2, L, p}.
void recycle_state_layout(pseudo_ctx *h, const pseudo_opts *o, int64_t npts, int64_t *out) {
    char *const base = (char *)4096;
    Carver c(base, (size_t)1 << 62);
    RecyLayout R;
    recy_layout(h, o, npts, c, R, o->io_host != 0);
    auto off = [&](const void *p) { return (int64_t)((const char *)p - base); };
    const int64_t v[11] = {R.L, R.KM, R.Ld, off(R.V), off(R.W1), off(R.W3), off(R.W4), off(R.H1), off(R.H2),
                           off(R.Lf), off(R.p)};
    for (int i = 0; i < 11; ++i) out[i] = v[i];
}

// Batch-zigzag visiting order (Sec. 2.3, eq. (batch)): column batches of b
// points, batch-rows in a row-wise zigzag, each batch visited vertically.
static std::vector<int> batch_zigzag(int64_t npts, int nx, int ny, int b) {
    std::vector<int> ord;
    ord.reserve(npts);
    if (nx <= 0 || ny <= 0) {
        for (int64_t i = 0; i < npts; ++i) ord.push_back((int)i);
        return ord;
    }
    const int nbr = (ny + b - 1) / b;
    for (int t = 0; t < nbr; ++t) {
        for (int q = 0; q < nx; ++q) {
            const int ix = (t % 2 == 0) ? q : nx - 1 - q;
            for (int iy = t * b; iy < std::min(ny, t * b + b); ++iy) ord.push_back(iy * nx + ix);
        }
    }
    return ord;
}

// Side of the smallest 2^q x 2^q square holding an nx x ny grid.
static int64_t curve_side(int nx, int ny) {
    int64_t side = 1;
    while (side < std::max(nx, ny)) side <<= 1;
    return side;
}

// Hilbert order (Sec. 5): the curve of side 2^q that runs from (0, 0) to
// (side - 1, 0), points outside the grid skipped.  Position d on the curve is
// mapped to (x, y) two bits at a time, from the smallest sub-square up: the
// two bits pick the quadrant, and the part already built is transposed (lower
// left) or reflected in the anti-diagonal (lower right) before being moved
// into it.
static std::vector<int> hilbert_order(int nx, int ny) {
    const int64_t side = curve_side(nx, ny);
    std::vector<int> ord;
    ord.reserve((size_t)nx * ny);
    for (int64_t d = 0; d < side * side; ++d) {
        int64_t x = 0, y = 0, t = d;
        for (int64_t s = 1; s < side; s <<= 1, t >>= 2) {
            const int64_t qx = (t >> 1) & 1, qy = (t ^ qx) & 1;
            if (qy == 0) {
                if (qx == 1) {
                    x = s - 1 - x;
                    y = s - 1 - y;
                }
                std::swap(x, y);
            }
            x += s * qx;
            y += s * qy;
        }
        if (x < nx && y < ny) ord.push_back((int)(y * nx + x));
    }
    return ord;
}

// Morton (Z-order, Sec. 5): points sorted by the interleaving of the bits of
// ix (even bit positions) and iy (odd positions).
static std::vector<int> morton_order(int nx, int ny) {
    auto spread = [](uint64_t v) {
        uint64_t r = 0;
        for (int b = 0; b < 32; ++b) r |= ((v >> b) & 1ull) << (2 * b);
        return r;
    };
    std::vector<std::pair<uint64_t, int>> key;
    key.reserve((size_t)nx * ny);
    for (int iy = 0; iy < ny; ++iy)
        for (int ix = 0; ix < nx; ++ix) key.emplace_back(spread(ix) | (spread(iy) << 1), iy * nx + ix);
    std::sort(key.begin(), key.end());
    std::vector<int> ord(key.size());
    for (size_t i = 0; i < key.size(); ++i) ord[i] = key[i].second;
    return ord;
}

// The recycling path's visiting order for the chosen traversal.
static std::vector<int> grid_order(int64_t npts, int nx, int ny, int b, int traversal) {
    if (nx > 0 && ny > 0) {
        if (traversal == PSEUDO_TRAVERSE_HILBERT) return hilbert_order(nx, ny);
        if (traversal == PSEUDO_TRAVERSE_MORTON) return morton_order(nx, ny);
    }
    return batch_zigzag(npts, nx, ny, b);
}

// FP64-corrected inverse-iteration polish of cnt unit vectors U (n x cnt)
// with shifts zc, followed by the Rayleigh quotient s2 and residual rr.
static cudaError_t polish_and_rq(pseudo_ctx *h, RecyLayout &R, int cnt, int polish, int max_ir,
                                 const std::vector<int> &items_h, cudaStream_t s) {
    const int n = h->n;
    cudaError_t e = cudaSuccess;
    if (polish) {
        IRBufs ib{R.R64, R.D32, R.rn2, R.mask, R.need, R.perm, (float2 *)R.xs, R.xh, R.xl, R.oz};
        IRPlan plan;
        {
            std::vector<double> xi((size_t)R.B * LB_MAXM), sg(cnt);
            std::vector<double2> zr(R.B), zh(cnt);
            cudaMemcpyAsync(xi.data(), R.xi, xi.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(zr.data(), R.zr, zr.size() * sizeof(double2), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            for (int t = 0; t < cnt; ++t) {
                const double x1 = xi[(size_t)items_h[t] * LB_MAXM];
                sg[t] = x1 > 0.0 ? 1.0 / x1 : 0.0;
                zh[t] = zr[items_h[t]];
            }
            ir_plan(h, sg, zh, max_ir, ib, plan, s);
        }
        if ((e = ir_solve_cols(h, ib, 1, R.zc, cnt, R.U, R.X64, plan, s)) != cudaSuccess) return e;
        cudaMemcpyAsync(R.B64, R.X64, (size_t)n * cnt * sizeof(double2), cudaMemcpyDeviceToDevice, s);
        if ((e = ir_solve_cols(h, ib, 0, R.zc, cnt, R.B64, R.X64, plan, s)) != cudaSuccess) return e;
        launch_normalize(R.X64, n, cnt, nullptr, s);
        cudaMemcpyAsync(R.U, R.X64, (size_t)n * cnt * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    }
    int k1 = kp_begin(h, s);
    trmv_hp(h, R.fp32, 0, nullptr, R.zc, cnt, R.U, cnt, nullptr, cnt, R.Y, cnt, 0, s, R.xh, R.xl, R.oz);
    trmv_hp(h, R.fp32, 1, nullptr, R.zc, cnt, R.Y, cnt, nullptr, cnt, R.NX, cnt, 0, s, R.xh, R.xl, R.oz);
    kp_end(h, k1, R.fp32 ? PSEUDO_K_TRMV_DS : PSEUDO_K_TRMV64, 2 * tri_flops(n, cnt), 2 * tri_bytes(n, cnt, 16, 16, 2), s);
    h->stats.mv_M_fp64_refine += 2 * (int64_t)cnt;
    launch_rq_residual(R.U, R.Y, R.NX, n, cnt, nullptr, R.s2, R.rr, s);
    return cudaGetLastError();
}

// Solve on the listed columns of buf (FP64 buffer of width Wd) in place:
// adjoint -> (T - zI)^{-H}, else (T - zI)^{-1}.  Mixed precision copies the
// columns (scaled per item by 1/scale) to FP32, solves, and copies back.
static cudaError_t solve_listed(pseudo_ctx *h, RecyLayout &R, double2 *buf, int ncols, int adjoint,
                                const double *scale, cudaStream_t s) {
    if (ncols <= 0) return cudaSuccess;
    const int n = h->n, r3 = 3 * R.r;
    if (!R.fp32) {
        const int k0 = kp_begin(h, s);
        cudaError_t e = launch_trsv64(adjoint ? h->L64 : h->U64, n, h->n_pad, adjoint, R.cols, R.zcol, ncols, nullptr,
                                      buf, R.Wd, (double2 *)R.xs, s);
        kp_end(h, k0, PSEUDO_K_TRSV64, tri_flops(n, ncols), tri_bytes(n, ncols, 16, 16, 2), s);
        return e;
    }
    launch_copy_listed<double2, float2>(buf, R.SB32, n, R.Wd, R.cols, ncols, 0, 0, r3, scale, LB_MAXM, 1, s);
    const int k0 = kp_begin(h, s);
    cudaError_t e = solve32(h, adjoint, R.cols, R.zcol, ncols, nullptr,
                                  R.SB32, R.Wd, (float2 *)R.xs, s);
    kp_end(h, k0, PSEUDO_K_TRSV32, tri_flops(n, ncols), tri_bytes(n, ncols, 8, 8, 2), s);
    if (e != cudaSuccess) return e;
    launch_copy_listed<float2, double2>(R.SB32, buf, n, R.Wd, R.cols, ncols, 0, 0, r3, scale, LB_MAXM, 0, s);
    return cudaGetLastError();
}

// Gram per listed item; the output of every round point is cleared first
// (the kernel accumulates slices with atomics).
static void gram_items(RecyLayout &R, TSView A, int ka, TSView B, int kb, int n, int nact, double2 *G, int64_t gstride,
                       cudaStream_t s) {
    cudaMemsetAsync(G, 0, sizeof(double2) * (size_t)gstride * R.B, s);
    launch_ts_gram(A, ka, B, kb, n, nact, R.items, G, gstride, false, s);
}

// Copy the listed item blocks: dst[:, j*3r + doff + c] = src[:, j*3r + soff + c], c < r
static void copy_item_blocks(RecyLayout &R, int n, const double2 *src, int soff, double2 *dst, int doff, int nact,
                             cudaStream_t s) {
    launch_make_cols(R.items, nact, R.r, soff, R.cols, s);
    launch_copy_listed<double2, double2>(src, dst, n, R.Wd, R.cols, nact * R.r, 0, doff - soff, 3 * R.r, nullptr, 0, 0,
                                         s);
}

// LOBPCG-SVD for the rejected points listed in R.items[0..nr) (Alg. SM1.2).
static int lobpcg_refine(pseudo_ctx *h, const pseudo_opts *o, RecyLayout &R, int nr, std::vector<int> &items_h,
                         cudaStream_t s) {
    const int n = h->n, r = R.r, r3 = 3 * r, MM = LB_MAXM * LB_MAXM;
    const int64_t ld = R.Wd;
    cudaError_t e;
    std::vector<int> act(items_h.begin(), items_h.begin() + nr);
    int nact = nr;
    auto upload_items = [&]() {
        cudaMemcpyAsync(R.items, act.data(), nact * sizeof(int), cudaMemcpyHostToDevice, s);
    };
    upload_items();
    const TSView Sx = tsv(R.S, ld, r3), CSx = tsv(R.CS, ld, r3);
    // orthonormalise X0 (CholeskyQR twice)
    for (int pass = 0; pass < 2; ++pass) {
        gram_items(R, Sx, r, Sx, r, n, nact, R.Gr, (int64_t)r * r, s);
        launch_chol_rinv(R.Gr, r, nact, R.items, R.Rinv, s);
        launch_ts_mul(Sx, r, R.Rinv, (int64_t)r * r, tsv(R.Sn, ld, r3), r, n, nact, R.items, 0.0, 1.0, s);
        copy_item_blocks(R, n, R.Sn, 0, R.S, 0, nact, s);
    }
    // CX0 = C X0
    copy_item_blocks(R, n, R.S, 0, R.CS, 0, nact, s);
    launch_make_cols(R.items, nact, r, 0, R.cols, s);
    if ((e = solve_listed(h, R, R.CS, nact * r, 1, nullptr, s)) != cudaSuccess) return cuda_err(e, "lobpcg init solve");
    h->stats.sv_R += (int64_t)nact * r;
    // [~, R0] = qr(C X0), svd(R0) -> Xi, G ; X1 = X0 G, CX1 = CX0 G
    gram_items(R, CSx, r, CSx, r, n, nact, R.Gm, MM, s);
    launch_lob_rr(R.Gm, r, r, 0, nact, R.items, R.xi, R.GX, R.GP, s);
    launch_ts_mul(Sx, r, R.GX, MM, tsv(R.Sn, ld, r3), r, n, nact, R.items, 0.0, 1.0, s);
    launch_ts_mul(CSx, r, R.GX, MM, tsv(R.CSn, ld, r3), r, n, nact, R.items, 0.0, 1.0, s);
    copy_item_blocks(R, n, R.Sn, 0, R.S, 0, nact, s);
    copy_item_blocks(R, n, R.CSn, 0, R.CS, 0, nact, s);
    int np = 0;  // columns in P
    const double rt = o->rtol > 0.0 ? o->rtol : 0.0;
    // both precisions stop LOBPCG on the Kato--Temple-style estimate: the
    // refinement step after it improves the vector but cannot separate a
    // cluster of nearly equal singular values, so a point whose gap is too
    // small for the accuracy target must end flagged as not converged
    const double rtol_lob = rt;
    int it = 0;
    for (it = 0; it < o->maxiter_lobpcg && nact > 0; ++it) {
        // W = C^H (C X) - X Xi^2
        copy_item_blocks(R, n, R.CS, 0, R.Yb, 0, nact, s);
        launch_make_cols(R.items, nact, r, 0, R.cols, s);
        if ((e = solve_listed(h, R, R.Yb, nact * r, 0, R.xi, s)) != cudaSuccess) return cuda_err(e, "lobpcg solve");
        h->stats.sv_R += (int64_t)nact * r;
        cudaMemsetAsync(R.conv, 0, R.B * sizeof(int), s);
        launch_lob_resid(R.S, R.Yb, n, ld, r, nact, R.items, R.xi, o->eta, rtol_lob, R.conv, R.wnorm, s);
        std::vector<int> convh(R.B);
        cudaMemcpyAsync(convh.data(), R.conv, R.B * sizeof(int), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_err(e, "lobpcg");
        std::vector<int> keep;
        for (int j : act)
            if (!convh[j]) keep.push_back(j);
        act.swap(keep);
        nact = (int)act.size();
        if (nact == 0) break;
        upload_items();
        h->stats.lobpcg_iters += 1;
        // W <- W - X (X^H W) - P (P^H W)   (K = I)
        const TSView Wv = tsv(R.S + r, ld, r3), Pv = tsv(R.S + 2 * r, ld, r3);
        for (int pass = 0; pass < 2; ++pass) {
            gram_items(R, Sx, r, Wv, r, n, nact, R.Gr, (int64_t)r * r, s);
            launch_ts_mul(Sx, r, R.Gr, (int64_t)r * r, Wv, r, n, nact, R.items, 1.0, -1.0, s);
            if (np) {
                gram_items(R, Pv, r, Wv, r, n, nact, R.Gr, (int64_t)r * r, s);
                launch_ts_mul(Pv, r, R.Gr, (int64_t)r * r, Wv, r, n, nact, R.items, 1.0, -1.0, s);
            }
        }
        // [W, ~] = qr(W): CholeskyQR twice
        for (int pass = 0; pass < 2; ++pass) {
            gram_items(R, Wv, r, Wv, r, n, nact, R.Gr, (int64_t)r * r, s);
            launch_chol_rinv(R.Gr, r, nact, R.items, R.Rinv, s);
            launch_ts_mul(Wv, r, R.Rinv, (int64_t)r * r, tsv(R.Sn + r, ld, r3), r, n, nact, R.items, 0.0, 1.0, s);
            copy_item_blocks(R, n, R.Sn, r, R.S, r, nact, s);
        }
        // CW = C W
        copy_item_blocks(R, n, R.S, r, R.CS, r, nact, s);
        launch_make_cols(R.items, nact, r, r, R.cols, s);
        if ((e = solve_listed(h, R, R.CS, nact * r, 1, nullptr, s)) != cudaSuccess) return cuda_err(e, "lobpcg solve");
        h->stats.sv_R += (int64_t)nact * r;
        // Rayleigh--Ritz-SVD on CS = [CX CW CP]
        const int m = r * 2 + np;
        gram_items(R, CSx, m, CSx, m, n, nact, R.Gm, MM, s);
        launch_lob_rr(R.Gm, m, r, 1, nact, R.items, R.xi, R.GX, R.GP, s);
        // X = S G_X, P = S G_P ; CX = CS G_X, CP = CS G_P
        launch_ts_mul(Sx, m, R.GX, MM, tsv(R.Sn, ld, r3), r, n, nact, R.items, 0.0, 1.0, s);
        launch_ts_mul(Sx, m, R.GP, MM, tsv(R.Sn + 2 * r, ld, r3), r, n, nact, R.items, 0.0, 1.0, s);
        launch_ts_mul(CSx, m, R.GX, MM, tsv(R.CSn, ld, r3), r, n, nact, R.items, 0.0, 1.0, s);
        launch_ts_mul(CSx, m, R.GP, MM, tsv(R.CSn + 2 * r, ld, r3), r, n, nact, R.items, 0.0, 1.0, s);
        copy_item_blocks(R, n, R.Sn, 0, R.S, 0, nact, s);
        copy_item_blocks(R, n, R.Sn, 2 * r, R.S, 2 * r, nact, s);
        copy_item_blocks(R, n, R.CSn, 0, R.CS, 0, nact, s);
        copy_item_blocks(R, n, R.CSn, 2 * r, R.CS, 2 * r, nact, s);
        np = r;
    }
    // points still active hit the iteration cap
    std::vector<int> nf(R.B, 0);
    for (int j : act) nf[j] = PSEUDO_PT_NOT_CONVERGED;
    cudaMemcpyAsync(R.nflag, nf.data(), R.B * sizeof(int), cudaMemcpyHostToDevice, s);
    h->stats.n_not_converged += nact;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_err(e, "lobpcg end");
    return nact;
}

// updateRecy for the lanes of one slot (Alg. 2).  slots: (lane, round point)
static int update_slot(pseudo_ctx *h, const pseudo_opts *o, RecyLayout &R, const std::vector<int> &sl_lane,
                       const std::vector<int> &sl_item, cudaStream_t s) {
    const int n = h->n, r = R.r, KM = R.KM, Ld = R.Ld;
    int nu = (int)sl_lane.size();
    if (nu == 0) return 0;
    cudaError_t e;
    cudaMemcpyAsync(R.slot_lanes, sl_lane.data(), nu * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(R.slot_items, sl_item.data(), nu * sizeof(int), cudaMemcpyHostToDevice, s);
    const TSView Vl = tsv(R.V, Ld, KM, R.slot_lanes), W1l = tsv(R.W1, Ld, KM, R.slot_lanes);
    const TSView Xs = tsv(R.Xst, (int64_t)R.L * r, r), X2 = tsv(R.Xt2, (int64_t)R.L * r, r);
    // X of each slot's refined point -> Xst
    launch_copy_block(tsv(R.S, R.Wd, 3 * r, R.slot_items), Xs, n, r, nu, nullptr, s);
    // c = V^H X (first column gives the rho's), ||x_1||
    launch_ts_gram(Vl, KM, Xs, r, n, nu, nullptr, R.Cc, (int64_t)KM * r, true, s);
    launch_ts_gram(Xs, r, Xs, r, n, nu, nullptr, R.gx, (int64_t)r * r, true, s);
    cudaMemsetAsync(R.nskip, 0, sizeof(int), s);
    launch_upd_decide(R.slot_lanes, nu, R.p, r, KM, KM / r, o->omega, R.Cc, R.gx, R.lout, R.kk, R.nskip, s);
    std::vector<int> lh(nu), kh(nu);
    cudaMemcpyAsync(lh.data(), R.lout, nu * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(kh.data(), R.kk, nu * sizeof(int), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_err(e, "update decide");
    // keep only appending slots (compact on the host, re-upload)
    std::vector<int> al, ai, ak, aslot;
    for (int u = 0; u < nu; ++u)
        if (lh[u] >= 0) { al.push_back(sl_lane[u]); ai.push_back(sl_item[u]); ak.push_back(kh[u]); aslot.push_back(u); }
    // drop leading blocks (uses lout of the original slot order)
    launch_upd_shift(R.V, R.W1, R.W3, R.W4, n, Ld, R.H1, R.H2, R.Lf, R.Cc, KM, r, R.slot_lanes, nu, R.p, R.lout, s);
    const int na = (int)al.size();
    if (na == 0) return 0;
    if (na != nu) {
        // compact per-slot arrays Cc (KM x r) and Xst columns to the appending slots
        std::vector<int> ident(na);
        for (int t = 0; t < na; ++t) ident[t] = aslot[t];
        cudaMemcpyAsync(R.slot_items, ident.data(), na * sizeof(int), cudaMemcpyHostToDevice, s);
        launch_copy_block(tsv(R.Xst, (int64_t)R.L * r, r, R.slot_items), X2, n, r, na, nullptr, s);
        launch_copy_block(X2, Xs, n, r, na, nullptr, s);
        cudaMemcpyAsync(R.C2, R.Cc, (size_t)nu * KM * r * sizeof(double2), cudaMemcpyDeviceToDevice, s);
        for (int t = 0; t < na; ++t)
            cudaMemcpyAsync(R.Cc + (size_t)t * KM * r, R.C2 + (size_t)aslot[t] * KM * r, KM * r * sizeof(double2),
                            cudaMemcpyDeviceToDevice, s);
        nu = na;
    }
    cudaMemcpyAsync(R.slot_lanes, al.data(), nu * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(R.kk, ak.data(), nu * sizeof(int), cudaMemcpyHostToDevice, s);
    // BCGS2 of X against the kept V: X -= V U (U = kept rows of c), twice
    launch_ts_mul(Vl, KM, R.Cc, (int64_t)KM * r, Xs, r, n, nu, nullptr, 1.0, -1.0, s);
    launch_ts_gram(Vl, KM, Xs, r, n, nu, nullptr, R.C2, (int64_t)KM * r, true, s);
    launch_ts_mul(Vl, KM, R.C2, (int64_t)KM * r, Xs, r, n, nu, nullptr, 1.0, -1.0, s);
    launch_upd_add(R.Cc, R.C2, KM * r, nu, s);
    // V_new U_new = X: CholeskyQR twice (R = R2 R1), V_new written into the lane's block
    launch_ts_gram(Xs, r, Xs, r, n, nu, nullptr, R.gx, (int64_t)r * r, true, s);
    launch_upd_chol(R.gx, r, nu, nullptr, R.Rn, R.Rni, s);
    launch_ts_mul(Xs, r, R.Rni, (int64_t)r * r, X2, r, n, nu, nullptr, 0.0, 1.0, s);
    launch_ts_gram(X2, r, X2, r, n, nu, nullptr, R.gx, (int64_t)r * r, true, s);
    launch_upd_chol(R.gx, r, nu, nullptr, R.R2, R.R2i, s);
    const TSView Vnew = tsv(R.V, Ld, KM, R.slot_lanes, R.kk), W1new = tsv(R.W1, Ld, KM, R.slot_lanes, R.kk);
    launch_ts_mul(X2, r, R.R2i, (int64_t)r * r, Vnew, r, n, nu, nullptr, 0.0, 1.0, s);
    launch_small_matmul(R.R2, R.Rn, R.Rf, r, nu, s);
    // W1+ = T V+, W4+ = T^H V+, W3+ = T^H W1+  (3r products with M per update)
    note_launch(); lane_cols_kernel<<<(nu * r + 127) / 128, 128, 0, s>>>(R.slot_lanes, R.kk, nu, r, KM, R.ucols);
    const int k1 = kp_begin(h, s);
    trmv_hp(h, R.fp32, 0, R.ucols, nullptr, nu * r, R.V, Ld, nullptr, Ld, R.W1, Ld, 0, s, R.xh, R.xl, R.oz);
    trmv_hp(h, R.fp32, 1, R.ucols, nullptr, nu * r, R.V, Ld, nullptr, Ld, R.W4, Ld, 0, s, R.xh, R.xl, R.oz);
    trmv_hp(h, R.fp32, 1, R.ucols, nullptr, nu * r, R.W1, Ld, nullptr, Ld, R.W3, Ld, 0, s, R.xh, R.xl, R.oz);
    kp_end(h, k1, R.fp32 ? PSEUDO_K_TRMV_DS : PSEUDO_K_TRMV64, 3 * tri_flops(n, nu * r),
           3 * tri_bytes(n, nu * r, 16, 16, 2), s);
    h->stats.mv_M += 3 * (int64_t)nu * r;
    // new blocks of H1 = W1^H W1 and H2 = W1^H V
    launch_ts_gram(W1l, KM, W1new, r, n, nu, nullptr, R.Hc1, (int64_t)KM * r, true, s);
    launch_ts_gram(W1l, KM, Vnew, r, n, nu, nullptr, R.Hc2, (int64_t)KM * r, true, s);
    launch_ts_gram(W1new, r, Vl, KM, n, nu, nullptr, R.Hr2, (int64_t)r * KM, true, s);
    // L, H1, H2 with the new block; restore the block lower-triangular L
    launch_upd_rotate(R.H1, R.H2, R.Lf, R.Qacc, R.Cc, R.Rf, R.Hc1, R.Hc2, R.Hr2, KM, r, R.slot_lanes, nu, R.p, R.kk, s);
    bool any_rot = false;
    for (int t = 0; t < nu; ++t) any_rot |= ak[t] > 0;
    if (any_rot) {
        const TSView Tl = tsv(R.Tmp, (int64_t)R.L * KM, KM);
        double2 *Ms[4] = {R.V, R.W1, R.W3, R.W4};
        for (int q = 0; q < 4; ++q) {
            const TSView Ml = tsv(Ms[q], Ld, KM, R.slot_lanes);
            launch_ts_mul(Ml, KM, R.Qacc, (int64_t)KM * KM, Tl, KM, n, nu, nullptr, 0.0, 1.0, s);
            launch_copy_block(Tl, Ml, n, KM, nu, nullptr, s);
        }
    }
    h->stats.n_updates += nu;
    return (e = cudaGetLastError()) != cudaSuccess ? cuda_err(e, "update") : 0;
}

// Device time of the phases of Alg. 3 in the paper's breakdown (recySing,
// LOBPCG-SVD refinement, the refined points' values and residuals, updateRecy),
// plus the whole call: event pairs recorded on the stream around each phase
// and read at the next synchronisation of the stream, when they have passed.
// The events are released on every return path.
struct PhaseTimes {
    enum { RECYSING, REFINE, POLISH, UPDATE, TOTAL, NPH };
    static constexpr const char *name[NPH] = {"recySing", "lobpcgSvd", "refined values", "updateRecy",
                                              "psTriRecy"};
    cudaEvent_t ev[NPH][2] = {};
    bool pending[NPH] = {};
    bool ok = true;
    int open = 0;  // NVTX ranges pushed and not yet popped
    double *acc[NPH];
    explicit PhaseTimes(pseudo_stats_t &st)
        : acc{&st.ms_recysing, &st.ms_refine, &st.ms_polish, &st.ms_update, &st.ms_total} {
        for (auto &pr : ev)
            for (auto &e : pr)
                if (cudaEventCreate(&e) != cudaSuccess) { e = nullptr; ok = false; }
    }
    ~PhaseTimes() {
        for (auto &pr : ev)
            for (auto &e : pr)
                if (e) cudaEventDestroy(e);
        while (open > 0) { nvtxRangePop(); --open; }  // a return inside a phase
    }
    // each phase is also a range on a profiler's NVTX timeline
    void begin(int ph, cudaStream_t s) {
        nvtxRangePushA(name[ph]);
        ++open;
        if (ok) cudaEventRecord(ev[ph][0], s);
    }
    void end(int ph, cudaStream_t s) {
        nvtxRangePop();
        --open;
        if (!ok) return;
        cudaEventRecord(ev[ph][1], s);
        pending[ph] = true;
    }
    // call only after the stream has been synchronised
    void collect() {
        for (int ph = 0; ph < NPH; ++ph) {
            if (!pending[ph]) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[ph][0], ev[ph][1]) == cudaSuccess) *acc[ph] += ms;
            pending[ph] = false;
        }
    }
};

int recycle_run(pseudo_ctx *h, const pseudo_opts *o, const GridIO &io, Carver &c, cudaStream_t s) {
    RecyLayout R;
    recy_layout(h, o, io.npts, c, R, io.on_host);
    if (c.overflow) return set_err(PSEUDO_ERR_WORKSPACE, "workspace too small");
    const int n = h->n;
    const int64_t npts = io.npts;
    cudaError_t e;
    PhaseTimes pt(h->stats);
    pt.begin(PhaseTimes::TOTAL, s);
    const double2 *zall = io.z;
    double *sig_all = io.sigma, *res_all = io.res;
    int32_t *flags_all = io.flags;
    uint32_t *member_all = io.member;
    if (io.on_host) {
        cudaMemcpyAsync(R.z_dev, io.z, npts * sizeof(double2), cudaMemcpyHostToDevice, s);
        zall = R.z_dev;
        sig_all = R.sig_dev;
        res_all = io.res ? R.res_dev : nullptr;
        flags_all = io.flags ? R.flags_dev : nullptr;
        member_all = io.member ? R.member_dev : nullptr;
    }
    if (io.neps > 0) cudaMemcpyAsync(R.eps, io.eps_host, io.neps * sizeof(double), cudaMemcpyHostToDevice, s);
    // state reset
    cudaMemsetAsync(R.V, 0, sizeof(double2) * (size_t)n * R.Ld, s);
    cudaMemsetAsync(R.W1, 0, sizeof(double2) * (size_t)n * R.Ld, s);
    cudaMemsetAsync(R.W3, 0, sizeof(double2) * (size_t)n * R.Ld, s);
    cudaMemsetAsync(R.W4, 0, sizeof(double2) * (size_t)n * R.Ld, s);
    cudaMemsetAsync(R.H1, 0, sizeof(double2) * (size_t)R.L * R.KM * R.KM, s);
    cudaMemsetAsync(R.H2, 0, sizeof(double2) * (size_t)R.L * R.KM * R.KM, s);
    cudaMemsetAsync(R.Lf, 0, sizeof(double2) * (size_t)R.L * R.KM * R.KM, s);
    cudaMemsetAsync(R.p, 0, sizeof(int) * R.L, s);
    // traversal and lane segments
    const int tb = std::max(1, o->batch_b);  // column-batch size of the traversal
    const std::vector<int> ord = grid_order(npts, o->grid_nx, o->grid_ny, tb, o->traversal);
    std::vector<int64_t> seg(R.L + 1);
    {
        const int64_t nbat = (npts + tb - 1) / tb;
        for (int l = 0; l <= R.L; ++l) seg[l] = std::min<int64_t>(npts, (nbat * l / R.L) * tb);
    }
    std::vector<int64_t> pos(seg.begin(), seg.end() - 1);
    std::vector<int> started(R.L, 0);
    const double eps_shift = o->eps_shift_rel * h->norm2 * h->norm2;
    const bool trace = getenv("PSEUDO_TRACE") != nullptr;  // per-round progress on stderr
    int64_t n_acc = 0, n_ref = 0;
    std::vector<int> gidx_r, lane_r, acc_h, rt_h, items_h;
    for (int round = 0;; ++round) {
        gidx_r.clear();
        lane_r.clear();
        for (int l = 0; l < R.L; ++l) {
            const int64_t take = started[l] ? R.b : 1;
            const int64_t end = std::min<int64_t>(seg[l + 1], pos[l] + take);
            for (int64_t q = pos[l]; q < end; ++q) { gidx_r.push_back(ord[q]); lane_r.push_back(l); }
            pos[l] = end;
        }
        const int np = (int)gidx_r.size();
        if (np == 0) break;
        cudaMemcpyAsync(R.ridx, gidx_r.data(), np * sizeof(int), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(R.lane_r, lane_r.data(), np * sizeof(int), cudaMemcpyHostToDevice, s);
        note_launch(); gather_z_kernel<<<(np + 127) / 128, 128, 0, s>>>(zall, R.ridx, np, R.zr);
        // 1. recySing for every point of the round
        RecySingLaunch rs;
        rs.n = n; rs.KM = R.KM; rs.r = R.r; rs.npts = np; rs.ldv = R.Ld;
        rs.V = R.V; rs.W1 = R.W1; rs.W3 = R.W3; rs.W4 = R.W4; rs.H1 = R.H1; rs.H2 = R.H2; rs.p = R.p;
        rs.z = R.zr; rs.lane = R.lane_r;
        rs.eps_shift = eps_shift; rs.tau = o->tau; rs.eta = o->eta; rs.rtol = o->rtol; rs.norm2 = h->norm2;
        rs.sigma = R.sig_r; rs.res = R.res_r; rs.xi2 = R.xi2_r; rs.w2 = R.w2_r; rs.accept = R.acc_r; rs.rt = R.rt_r;
        rs.CX = R.CX;
        {
            pt.begin(PhaseTimes::RECYSING, s);
            const int k0 = kp_begin(h, s);
            e = launch_recysing(rs, s);
            // per point: Y and its Gram (2k r + r^2 complex MACs per row, r = block size as a floor for r~),
            // two residual columns (8k per row), the k x k Jacobi (~9 k^3 real)
            const double kf = R.KM, rf = R.r;
            kp_end(h, k0, PSEUDO_K_RECYSING, np * (8.0 * n * (2 * kf * rf + rf * rf + 8 * kf) + 9 * kf * kf * kf),
                   (double)R.L * 4.0 * n * kf * 16.0, s);
            if (e != cudaSuccess) return cuda_err(e, "recySing");
            pt.end(PhaseTimes::RECYSING, s);
        }
        acc_h.assign(np, 0);
        rt_h.assign(np, 0);
        cudaMemcpyAsync(acc_h.data(), R.acc_r, np * sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(rt_h.data(), R.rt_r, np * sizeof(int), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_err(e, "recySing");
        pt.collect();
        for (int j = 0; j < np; ++j) h->stats.n_rtilde_capped += rt_h[j] > RTMAX ? 1 : 0;
        note_launch(); scatter_round_kernel<<<(np + 127) / 128, 128, 0, s>>>(nullptr, np, R.ridx, R.sig_r, R.res_r, PSEUDO_PT_ACCEPTED,
                                                              R.eps, io.neps, sig_all, res_all, flags_all, member_all,
                                                              nullptr);
        items_h.clear();
        for (int j = 0; j < np; ++j)
            if (!acc_h[j]) items_h.push_back(j);
        const int nr = (int)items_h.size();
        n_acc += np - nr;
        n_ref += nr;
        if (nr == 0) continue;
        // 2. refinement: start from X~ = V C_X (or a seeded random block for an empty subspace)
        pt.begin(PhaseTimes::REFINE, s);
        cudaMemcpyAsync(R.items, items_h.data(), nr * sizeof(int), cudaMemcpyHostToDevice, s);
        launch_expand_shift(R.zr, R.B, R.r, R.zcol, s);
        {
            std::vector<int> cold, warm;
            for (int j : items_h) (started[lane_r[j]] ? warm : cold).push_back(j);
            if (!warm.empty()) {
                cudaMemcpyAsync(R.items, warm.data(), warm.size() * sizeof(int), cudaMemcpyHostToDevice, s);
                launch_ts_mul(tsv(R.V, R.Ld, R.KM, R.lane_r), R.KM, R.CX, (int64_t)R.KM * R.r, tsv(R.S, R.Wd, 3 * R.r),
                              R.r, n, (int)warm.size(), R.items, 0.0, 1.0, s);
            }
            if (!cold.empty()) {
                cudaMemcpyAsync(R.items, cold.data(), cold.size() * sizeof(int), cudaMemcpyHostToDevice, s);
                dim3 g(32, (unsigned)cold.size());
                note_launch(); rand_block_kernel<<<g, 256, 0, s>>>(R.S, n, R.Wd, R.r, R.items, (int)cold.size(), R.ridx,
                                                    o->seed + 7919ull * round);
            }
        }
        const int64_t it0 = h->stats.lobpcg_iters;
        const int nbad = lobpcg_refine(h, o, R, nr, items_h, s);
        if (trace)
            fprintf(stderr, "[pseudo] round %d: %d points, %d refined, %lld LOBPCG iterations, %d unconverged\n", round,
                    np, nr, (long long)(h->stats.lobpcg_iters - it0), nbad);
        if (nbad < 0) return nbad;
        pt.end(PhaseTimes::REFINE, s);
        // 3. sigma and residual of the refined points (polished in mixed precision)
        pt.begin(PhaseTimes::POLISH, s);
        cudaMemcpyAsync(R.items, items_h.data(), nr * sizeof(int), cudaMemcpyHostToDevice, s);
        note_launch(); x1_gather_kernel<<<(nr + 31) / 32, 256, 0, s>>>(R.S, R.Wd, R.r, R.items, nr, n, R.U, R.zr, R.zc, 0);
        launch_normalize(R.U, n, nr, nullptr, s);
        if ((e = polish_and_rq(h, R, nr, R.fp32 ? 1 : 0, o->max_ir, items_h, s)) != cudaSuccess)
            return cuda_err(e, "polish");
        if (R.fp32) { note_launch(); x1_gather_kernel<<<(nr + 31) / 32, 256, 0, s>>>(R.S, R.Wd, R.r, R.items, nr, n, R.U, R.zr, R.zc, 1); }
        note_launch(); refined_values_kernel<<<(nr + 127) / 128, 128, 0, s>>>(R.items, nr, R.xi, R.s2, R.rr, R.zr, h->norm2,
                                                               R.fp32 ? 1 : 0, R.sig_r, R.res_r);
        note_launch(); scatter_round_kernel<<<(nr + 127) / 128, 128, 0, s>>>(R.items, nr, R.ridx, R.sig_r, R.res_r, PSEUDO_PT_REFINED,
                                                              R.eps, io.neps, sig_all, res_all, flags_all, member_all,
                                                              R.nflag);
        pt.end(PhaseTimes::POLISH, s);
        // 4. updateRecy per lane in visiting order: slot u = the u-th refined point of each lane
        pt.begin(PhaseTimes::UPDATE, s);
        std::vector<std::vector<int>> per_lane(R.L);
        for (int j : items_h) per_lane[lane_r[j]].push_back(j);
        size_t nslots = 0;
        for (auto &v : per_lane) nslots = std::max(nslots, v.size());
        for (size_t u = 0; u < nslots; ++u) {
            std::vector<int> sl, si;
            for (int l = 0; l < R.L; ++l)
                if (u < per_lane[l].size()) { sl.push_back(l); si.push_back(per_lane[l][u]); }
            const int rc = update_slot(h, o, R, sl, si, s);
            if (rc < 0) return rc;
        }
        pt.end(PhaseTimes::UPDATE, s);
        for (int l = 0; l < R.L; ++l)
            if (!per_lane[l].empty()) started[l] = 1;
    }
    if (io.on_host) {
        cudaMemcpyAsync(io.sigma, sig_all, npts * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (io.res) cudaMemcpyAsync(io.res, res_all, npts * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (io.flags) cudaMemcpyAsync(io.flags, flags_all, npts * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (io.member) cudaMemcpyAsync(io.member, member_all, npts * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    }
    pt.end(PhaseTimes::TOTAL, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_err(e, "pseudo_grid");
    pt.collect();
    h->stats.n_points += npts;
    h->stats.n_accepted += n_acc;
    h->stats.n_refined += n_ref;
    return PSEUDO_OK;
}

}  // namespace pseudo

extern "C" int pseudo_traversal_order(int64_t npts, int grid_nx, int grid_ny, int batch_b, int traversal,
                                      int32_t *order) {
    using namespace pseudo;
    if (npts < 0 || npts > INT32_MAX || grid_nx < 0 || grid_ny < 0 || batch_b < 1 || (npts > 0 && !order))
        return set_err(PSEUDO_ERR_ARG, "bad argument");
    if (traversal < PSEUDO_TRAVERSE_BATCH_ZIGZAG || traversal > PSEUDO_TRAVERSE_MORTON)
        return set_err(PSEUDO_ERR_ARG, "bad traversal %d", traversal);
    if (grid_nx > 0 && (int64_t)grid_nx * grid_ny != npts) return set_err(PSEUDO_ERR_ARG, "grid_nx * grid_ny != npts");
    const std::vector<int> ord = grid_order(npts, grid_nx, grid_ny, batch_b, traversal);
    std::copy(ord.begin(), ord.end(), order);
    return PSEUDO_OK;
}
