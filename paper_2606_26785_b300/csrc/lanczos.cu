// Shift-batched inverse Lanczos on N(z)^{-1} = (T - zI)^{-1} (T - zI)^{-H}
// (the EigTool core, Sec. 1): every column c of the batch is one grid point.
// One Lanczos step for all active columns is
//     w = (T - z I)^{-1} (T - z I)^{-H} q_j            (two multi-shift solves)
//     h = Q^H w, w -= Q h  (twice: classical Gram-Schmidt with full
//                           reorthogonalisation), alpha_j = Re h_j,
//     beta_j = ||w||, q_{j+1} = w / beta_j,
// followed by the largest eigenvalue theta of the tridiagonal T_j and the
// bound beta_j |s_j| on the Ritz residual; sigma = 1/sqrt(theta).
//
// Vectors live in row-major n x S arrays (row i of all columns contiguous).
// Kernels over columns use CTAs of 32 consecutive columns (lane = column,
// warps split the rows) so that loads are coalesced whatever subset of the
// columns is still active.
#include "common.cuh"
#include "internal.h"

namespace pseudo {

// ------------------------------------------------------- start vector
// Counter-based generator (SplitMix64 finaliser of seed + i): the start
// vector is the same for every grid point (no continuation between points).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void start_vector_kernel(double2 *v, int n, uint64_t seed) {
    __shared__ double ws[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        uint64_t a = splitmix64(seed * 0x100000001B3ull + 2ull * i);
        uint64_t b = splitmix64(seed * 0x100000001B3ull + 2ull * i + 1);
        double re = (double)(a >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        double im = (double)(b >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        v[i] = make_double2(re, im);
        s += re * re + im * im;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) ws[0] = 1.0 / sqrt(s);
    }
    __syncthreads();
    const double inv = ws[0];
    for (int i = threadIdx.x; i < n; i += blockDim.x) { v[i].x *= inv; v[i].y *= inv; }
}

template <typename real>
__global__ void bcast_start_kernel(const double2 *__restrict__ v, int n, int S, cx_t<real> *__restrict__ Q0) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * S) return;
    const int i = (int)(idx / S);
    Q0[idx] = mk<real>((real)v[i].x, (real)v[i].y);
}

// -------------------------------------------------- copy active columns
template <typename real>
__global__ void copy_cols_kernel(const cx_t<real> *__restrict__ src, cx_t<real> *__restrict__ dst, int n, int S,
                                 const int *__restrict__ active) {
    const int c = blockIdx.x * 32 + (threadIdx.x & 31);
    if (c >= S || active[c] != 1) return;
    for (int i = threadIdx.x >> 5; i < n; i += blockDim.x >> 5) dst[(int64_t)i * S + c] = src[(int64_t)i * S + c];
}

// --------------------------------------------------- orthogonalisation
constexpr int ORTH_WARPS = 8, TCH = 8;

template <typename real>
__global__ void __launch_bounds__(ORTH_WARPS * 32)
lanczos_orth_kernel(cx_t<real> *__restrict__ Q, int64_t qs, cx_t<real> *__restrict__ W, int n, int S, int j,
                    int mmax, const int *__restrict__ active, double *__restrict__ alpha,
                    double *__restrict__ beta) {
    using C = cx_t<real>;
    __shared__ double2 red[ORTH_WARPS][TCH][32];
    __shared__ double2 s_hj[32];
    __shared__ double s_nrm[ORTH_WARPS][32];
    __shared__ int any;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const bool on = (c < S) && active[c] == 1;
    if (threadIdx.x == 0) any = 0;
    if (threadIdx.x < 32) s_hj[threadIdx.x] = make_double2(0.0, 0.0);
    __syncthreads();
    if (on) any = 1;
    __syncthreads();
    if (!any) return;
    const int cc = on ? c : 0;
    for (int pass = 0; pass < 2; ++pass) {
        // h_t = q_t^H w for t = 0..j, in chunks of TCH vectors; then w -= q_t h_t
        for (int t0 = 0; t0 <= j; t0 += TCH) {
            // partial dot products in the vectors' own precision: FP32 vectors
            // get FP32 arithmetic (the FP64 units are 62x slower on this GPU)
            C acc[TCH];
#pragma unroll
            for (int u = 0; u < TCH; ++u) acc[u] = mk<real>(0, 0);
            if (on) {
                for (int i = warp; i < n; i += ORTH_WARPS) {
                    const C wv = W[(int64_t)i * S + cc];
#pragma unroll
                    for (int u = 0; u < TCH; ++u) {
                        if (t0 + u <= j) {
                            const C qv = Q[(int64_t)(t0 + u) * qs + (int64_t)i * S + cc];
                            cfma(acc[u], cconj(qv), wv);
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < TCH; ++u) red[warp][u][lane] = make_double2((double)acc[u].x, (double)acc[u].y);
            __syncthreads();
            if (warp == 0) {
                for (int u = 0; u < TCH && t0 + u <= j; ++u) {
                    double2 s = make_double2(0.0, 0.0);
                    for (int w = 0; w < ORTH_WARPS; ++w) { s.x += red[w][u][lane].x; s.y += red[w][u][lane].y; }
                    red[0][u][lane] = s;
                    if (t0 + u == j) { s_hj[lane].x += s.x; s_hj[lane].y += s.y; }
                }
            }
            __syncthreads();
            if (on) {
                C hc[TCH];
#pragma unroll
                for (int u = 0; u < TCH; ++u)
                    hc[u] = (t0 + u <= j) ? mk<real>((real)red[0][u][lane].x, (real)red[0][u][lane].y) : mk<real>(0, 0);
                for (int i = warp; i < n; i += ORTH_WARPS) {
                    C wv = W[(int64_t)i * S + cc];
#pragma unroll
                    for (int u = 0; u < TCH; ++u) {
                        if (t0 + u <= j) {
                            const C qv = Q[(int64_t)(t0 + u) * qs + (int64_t)i * S + cc];
                            cfms(wv, qv, hc[u]);
                        }
                    }
                    W[(int64_t)i * S + cc] = wv;
                }
            }
            __syncthreads();
        }
    }
    // beta = ||w||, q_{j+1} = w / beta
    real sp = 0;
    if (on)
        for (int i = warp; i < n; i += ORTH_WARPS) {
            const C wv = W[(int64_t)i * S + cc];
            sp += wv.x * wv.x + wv.y * wv.y;
        }
    s_nrm[warp][lane] = (double)sp;
    __syncthreads();
    if (warp == 0) {
        double t = 0.0;
        for (int w = 0; w < ORTH_WARPS; ++w) t += s_nrm[w][lane];
        s_nrm[0][lane] = sqrt(t);
    }
    __syncthreads();
    const double b = s_nrm[0][lane];
    if (on) {
        const double inv = b > 0.0 ? 1.0 / b : 0.0;
        for (int i = warp; i < n; i += ORTH_WARPS) {
            const C wv = W[(int64_t)i * S + cc];
            Q[(int64_t)(j + 1) * qs + (int64_t)i * S + cc] = mk<real>((real)(wv.x * inv), (real)(wv.y * inv));
        }
        if (warp == 0) {
            alpha[(int64_t)c * mmax + j] = s_hj[lane].x;
            beta[(int64_t)c * mmax + j] = b;
        }
    }
}

// ------------------------------------------------ tridiagonal eigen
// Sturm count: number of eigenvalues of the k x k symmetric tridiagonal
// (a, b) that are < x.
template <typename real>
__device__ int sturm_count(const real *a, const real *b, int k, real x, real pivmin) {
    int cnt = 0;
    real d = a[0] - x;
    if (fabs(d) < pivmin) d = -pivmin;
    if (d < 0) cnt++;
    for (int i = 1; i < k; ++i) {
        d = a[i] - x - b[i - 1] * b[i - 1] / d;
        if (fabs(d) < pivmin) d = -pivmin;
        if (d < 0) cnt++;
    }
    return cnt;
}

// eigenvalue number `idx` (0 = smallest) by bisection to a few units of the
// working precision
template <typename real>
__device__ real tridiag_eig(const real *a, const real *b, int k, int idx) {
    constexpr bool dbl = sizeof(real) == 8;
    const real eps = dbl ? (real)2.2e-16 : (real)1.2e-7;
    const real tiny = dbl ? (real)2.2250738585072014e-308 : (real)1.1754944e-38;
    real lo = a[0], hi = a[0];
    for (int i = 0; i < k; ++i) {
        real r = (i > 0 ? fabs(b[i - 1]) : (real)0) + (i < k - 1 ? fabs(b[i]) : (real)0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
    }
    const real scale = fmax(fabs(lo), fabs(hi));
    const real pivmin = fmax(tiny, (dbl ? (real)1e-300 : (real)1e-30) * scale * scale + tiny);
    for (int it = 0; it < 200; ++it) {
        real mid = (real)0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count<real>(a, b, k, mid, pivmin) > idx) hi = mid; else lo = mid;
        if (hi - lo <= eps * fmax(fabs(lo), fabs(hi))) break;
    }
    return (real)0.5 * (lo + hi);
}

// Eigenvector of the tridiagonal for eigenvalue lam by two steps of inverse
// iteration (tridiagonal LU with partial pivoting); result normalised.
template <typename real>
__device__ void tridiag_vec(const real *a, const real *b, int k, real lam, real *s, real *wk) {
    // wk layout: d (k), du (k), du2 (k), dl (k), piv as double (k)
    real *d = wk, *du = wk + k, *du2 = wk + 2 * k, *dl = wk + 3 * k, *pv = wk + 4 * k;
    const real tiny = sizeof(real) == 8 ? (real)(1e-300 + 1e-15 * fabs(lam)) : (real)(1e-30f + 1e-6f * fabs(lam));
    for (int i = 0; i < k; ++i) { s[i] = (real)1; }
    for (int rep = 0; rep < 2; ++rep) {
        for (int i = 0; i < k; ++i) { d[i] = a[i] - lam; du[i] = i < k - 1 ? b[i] : (real)0; dl[i] = i < k - 1 ? b[i] : (real)0; du2[i] = 0; pv[i] = 0; }
        for (int i = 0; i < k - 1; ++i) {
            if (fabs(d[i]) >= fabs(dl[i])) {
                if (fabs(d[i]) < tiny) d[i] = tiny;
                real f = dl[i] / d[i];
                dl[i] = f;
                d[i + 1] -= f * du[i];
                pv[i] = 0;
            } else {
                real f = d[i] / dl[i];
                d[i] = dl[i];
                dl[i] = f;
                real tmp = du[i];
                du[i] = d[i + 1];
                d[i + 1] = tmp - f * d[i + 1];
                if (i < k - 2) { du2[i] = du[i + 1]; du[i + 1] = -f * du[i + 1]; }
                pv[i] = 1;
            }
        }
        if (fabs(d[k - 1]) < tiny) d[k - 1] = tiny;
        // forward: apply L^{-1} P
        for (int i = 0; i < k - 1; ++i) {
            if (pv[i] != (real)0) { real t = s[i]; s[i] = s[i + 1]; s[i + 1] = t - dl[i] * s[i]; }
            else s[i + 1] -= dl[i] * s[i];
        }
        // backward: U^{-1}
        s[k - 1] /= d[k - 1];
        if (k > 1) s[k - 2] = (s[k - 2] - du[k - 2] * s[k - 1]) / d[k - 2];
        for (int i = k - 3; i >= 0; --i) s[i] = (s[i] - du[i] * s[i + 1] - du2[i] * s[i + 2]) / d[i];
        real nr = 0;
        for (int i = 0; i < k; ++i) nr += s[i] * s[i];
        nr = (real)1 / sqrt(nr);
        for (int i = 0; i < k; ++i) s[i] *= nr;
    }
}

// For every active column after step j: theta_max, gap and convergence.
__global__ void lanczos_tridiag_kernel(int S, int j, int mmax, const double *__restrict__ alpha,
                                       const double *__restrict__ beta, int *__restrict__ active,
                                       double *__restrict__ theta, double *__restrict__ svec,
                                       int *__restrict__ nsteps, double tol_q, double tol_floor,
                                       int final_step) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= S || !active[c]) return;
    const int k = j + 1;
    double a[LANCZOS_MMAX], b[LANCZOS_MMAX], s[LANCZOS_MMAX], wk[5 * LANCZOS_MMAX];
    for (int i = 0; i < k; ++i) { a[i] = alpha[(int64_t)c * mmax + i]; b[i] = beta[(int64_t)c * mmax + i]; }
    const double th1 = tridiag_eig<double>(a, b, k, k - 1);
    const double th2 = k > 1 ? tridiag_eig<double>(a, b, k, k - 2) : 0.0;
    tridiag_vec<double>(a, b, k, th1, s, wk);
    const double rb = fabs(b[k - 1] * s[k - 1]);  // ||N^{-1} u - theta u||
    const double gap = fmax(th1 - th2, 1e-300);
    const double est = rb * rb / (th1 * gap);     // relative error bound on theta
    const bool breakdown = b[k - 1] <= 1e-300 * th1;
    const bool conv = breakdown || est <= tol_q || rb <= tol_floor * th1;
    theta[c] = th1;
    nsteps[c] = k;
    for (int i = 0; i < k; ++i) svec[(int64_t)c * mmax + i] = s[i];
    if (conv || final_step) active[c] = conv ? 0 : -1;  // -1: stopped unconverged
}

// Active list: cols[] = indices with active[c] == 1, count in *cnt.  One CTA.
__global__ void compact_active_kernel(const int *__restrict__ active, int S, int *__restrict__ cols, int *cnt) {
    __shared__ int base;
    __shared__ int wsum[32];
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < S; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const int f = (c < S && active[c] == 1) ? 1 : 0;
        const unsigned m = __ballot_sync(0xffffffffu, f);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) wsum[warp] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { int t = wsum[w]; wsum[w] = acc; acc += t; }
        }
        __syncthreads();
        if (f) cols[base + wsum[warp] + __popc(m & ((1u << lane) - 1u))] = c;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) base += wsum[warp] + __popc(m);
        __syncthreads();
    }
    if (threadIdx.x == 0) *cnt = base;
}

// Ritz vector u_c = sum_t s_t q_t (FP64 out), normalised.
template <typename real>
__global__ void __launch_bounds__(ORTH_WARPS * 32)
ritz_vector_kernel(const cx_t<real> *__restrict__ Q, int64_t qs, int n, int S, int mmax,
                   const double *__restrict__ svec, const int *__restrict__ nsteps, double2 *__restrict__ U,
                   const int *__restrict__ mask) {
    __shared__ double s_nrm[ORTH_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const bool on = c < S && (mask == nullptr || mask[c]);
    const int k = on ? nsteps[c] : 0;
    double s = 0.0;
    for (int i = warp; i < n; i += ORTH_WARPS) {
        if (!on) break;
        double ur = 0.0, ui = 0.0;
        for (int t = 0; t < k; ++t) {
            const double st = svec[(int64_t)c * mmax + t];
            const cx_t<real> qv = Q[(int64_t)t * qs + (int64_t)i * S + c];
            ur += st * qv.x; ui += st * qv.y;
        }
        U[(int64_t)i * S + c] = make_double2(ur, ui);
        s += ur * ur + ui * ui;
    }
    s_nrm[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
        double t = 0.0;
        for (int w = 0; w < ORTH_WARPS; ++w) t += s_nrm[w][lane];
        s_nrm[0][lane] = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
    }
    __syncthreads();
    const double inv = s_nrm[0][lane];
    if (on)
        for (int i = warp; i < n; i += ORTH_WARPS) { double2 v = U[(int64_t)i * S + c]; v.x *= inv; v.y *= inv; U[(int64_t)i * S + c] = v; }
}

// ------------------------------------------------------------ launchers
void launch_start_vector(double2 *v, int n, uint64_t seed, cudaStream_t s) {
    note_launch(); start_vector_kernel<<<1, 1024, 0, s>>>(v, n, seed);
}
template <typename real>
void launch_bcast_start(const double2 *v, int n, int S, cx_t<real> *Q0, cudaStream_t s) {
    int64_t tot = (int64_t)n * S;
    note_launch(); bcast_start_kernel<real><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(v, n, S, Q0);
}
template <typename real>
void launch_copy_cols(const cx_t<real> *src, cx_t<real> *dst, int n, int S, const int *active, cudaStream_t s) {
    note_launch(); copy_cols_kernel<real><<<(S + 31) / 32, 256, 0, s>>>(src, dst, n, S, active);
}
template <typename real>
void launch_lanczos_orth(cx_t<real> *Q, int64_t qs, cx_t<real> *W, int n, int S, int j, int mmax, const int *active,
                         double *alpha, double *beta, cudaStream_t s) {
    note_launch(); lanczos_orth_kernel<real><<<(S + 31) / 32, ORTH_WARPS * 32, 0, s>>>(Q, qs, W, n, S, j, mmax, active, alpha, beta);
}
void launch_lanczos_tridiag(int S, int j, int mmax, const double *alpha, const double *beta, int *active,
                            double *theta, double *svec, int *nsteps, double tol_q, double tol_floor, int final_step,
                            cudaStream_t s) {
    note_launch(); lanczos_tridiag_kernel<<<(S + 63) / 64, 64, 0, s>>>(S, j, mmax, alpha, beta, active, theta, svec, nsteps, tol_q,
                                                        tol_floor, final_step);
}
void launch_compact_active(const int *active, int S, int *cols, int *cnt, cudaStream_t s) {
    note_launch(); compact_active_kernel<<<1, 1024, 0, s>>>(active, S, cols, cnt);
}
template <typename real>
void launch_ritz_vector(const cx_t<real> *Q, int64_t qs, int n, int S, int mmax, const double *svec, const int *nsteps,
                        double2 *U, const int *mask, cudaStream_t s) {
    note_launch(); ritz_vector_kernel<real><<<(S + 31) / 32, ORTH_WARPS * 32, 0, s>>>(Q, qs, n, S, mmax, svec, nsteps, U, mask);
}

template void launch_bcast_start<float>(const double2 *, int, int, float2 *, cudaStream_t);
template void launch_bcast_start<double>(const double2 *, int, int, double2 *, cudaStream_t);
template void launch_copy_cols<float>(const float2 *, float2 *, int, int, const int *, cudaStream_t);
template void launch_copy_cols<double>(const double2 *, double2 *, int, int, const int *, cudaStream_t);
template void launch_lanczos_orth<float>(float2 *, int64_t, float2 *, int, int, int, int, const int *, double *, double *, cudaStream_t);
template void launch_lanczos_orth<double>(double2 *, int64_t, double2 *, int, int, int, int, const int *, double *, double *, cudaStream_t);
template void launch_ritz_vector<float>(const float2 *, int64_t, int, int, int, const double *, const int *, double2 *, const int *, cudaStream_t);
template void launch_ritz_vector<double>(const double2 *, int64_t, int, int, int, const double *, const int *, double2 *, const int *, cudaStream_t);

}  // namespace pseudo

// ===================== continuous batching (slots refilled on convergence)
// A wave of S slots runs Lanczos recurrences that start and finish at
// different global iterations: every slot c carries its own step jv[c].
// active[c]: 1 running, 2 finished this iteration (to harvest), 3 empty
// (to fill), 0 idle (no points left).
namespace pseudo {

// W[:, c] = Q[jv[c]][:, c] for running slots
template <typename real>
__global__ void slot_copy_kernel(const cx_t<real> *__restrict__ Q, int64_t qs, cx_t<real> *__restrict__ W, int n,
                                 int S, const int *__restrict__ jv, const int *__restrict__ active) {
    const int c = blockIdx.x * 32 + (threadIdx.x & 31);
    if (c >= S || active[c] != 1) return;
    const cx_t<real> *q = Q + (int64_t)jv[c] * qs;
    for (int i = threadIdx.x >> 5; i < n; i += blockDim.x >> 5) W[(int64_t)i * S + c] = q[(int64_t)i * S + c];
}

// Reorthogonalise w against q_0..q_{j_c} (classical Gram-Schmidt, `passes`
// times), alpha_j = Re(q_j^H w), beta_j = ||w||, q_{j+1} = w / beta.
template <typename real>
__global__ void __launch_bounds__(ORTH_WARPS * 32)
slot_orth_kernel(cx_t<real> *__restrict__ Q, int64_t qs, cx_t<real> *__restrict__ W, int n, int S,
                 const int *__restrict__ jv, int mmax, const int *__restrict__ active, double *__restrict__ alpha,
                 double *__restrict__ beta, int passes) {
    using C = cx_t<real>;
    __shared__ double2 red[ORTH_WARPS][TCH][32];
    __shared__ double2 s_hj[32];
    __shared__ double s_nrm[ORTH_WARPS][32];
    __shared__ int s_jmax;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const bool on = (c < S) && active[c] == 1;
    const int jc = on ? jv[c] : -1;
    if (threadIdx.x == 0) s_jmax = -1;
    if (threadIdx.x < 32) s_hj[threadIdx.x] = make_double2(0.0, 0.0);
    __syncthreads();
    if (warp == 0 && on) atomicMax(&s_jmax, jc);
    __syncthreads();
    const int jmax = s_jmax;
    if (jmax < 0) return;
    const int cc = on ? c : 0;
    for (int pass = 0; pass < passes; ++pass) {
        for (int t0 = 0; t0 <= jmax; t0 += TCH) {
            C acc[TCH];
#pragma unroll
            for (int u = 0; u < TCH; ++u) acc[u] = mk<real>(0, 0);
            if (on && t0 <= jc) {
                for (int i = warp; i < n; i += ORTH_WARPS) {
                    const C wv = W[(int64_t)i * S + cc];
#pragma unroll
                    for (int u = 0; u < TCH; ++u)
                        if (t0 + u <= jc) cfma(acc[u], cconj(Q[(int64_t)(t0 + u) * qs + (int64_t)i * S + cc]), wv);
                }
            }
#pragma unroll
            for (int u = 0; u < TCH; ++u) red[warp][u][lane] = make_double2((double)acc[u].x, (double)acc[u].y);
            __syncthreads();
            if (warp == 0) {
                for (int u = 0; u < TCH; ++u) {
                    double2 s = make_double2(0.0, 0.0);
                    for (int w = 0; w < ORTH_WARPS; ++w) { s.x += red[w][u][lane].x; s.y += red[w][u][lane].y; }
                    red[0][u][lane] = s;
                    if (on && t0 + u == jc) { s_hj[lane].x += s.x; s_hj[lane].y += s.y; }
                }
            }
            __syncthreads();
            if (on && t0 <= jc) {
                C hc[TCH];
#pragma unroll
                for (int u = 0; u < TCH; ++u)
                    hc[u] = (t0 + u <= jc) ? mk<real>((real)red[0][u][lane].x, (real)red[0][u][lane].y) : mk<real>(0, 0);
                for (int i = warp; i < n; i += ORTH_WARPS) {
                    C wv = W[(int64_t)i * S + cc];
#pragma unroll
                    for (int u = 0; u < TCH; ++u)
                        if (t0 + u <= jc) cfms(wv, Q[(int64_t)(t0 + u) * qs + (int64_t)i * S + cc], hc[u]);
                    W[(int64_t)i * S + cc] = wv;
                }
            }
            __syncthreads();
        }
    }
    real sp = 0;
    if (on)
        for (int i = warp; i < n; i += ORTH_WARPS) {
            const C wv = W[(int64_t)i * S + cc];
            sp += wv.x * wv.x + wv.y * wv.y;
        }
    s_nrm[warp][lane] = (double)sp;
    __syncthreads();
    if (warp == 0) {
        double t = 0.0;
        for (int w = 0; w < ORTH_WARPS; ++w) t += s_nrm[w][lane];
        s_nrm[0][lane] = sqrt(t);
    }
    __syncthreads();
    const double b = s_nrm[0][lane];
    if (on) {
        const double inv = b > 0.0 ? 1.0 / b : 0.0;
        for (int i = warp; i < n; i += ORTH_WARPS) {
            const C wv = W[(int64_t)i * S + cc];
            Q[(int64_t)(jc + 1) * qs + (int64_t)i * S + cc] = mk<real>((real)(wv.x * inv), (real)(wv.y * inv));
        }
        if (warp == 0) {
            alpha[(int64_t)c * mmax + jc] = s_hj[lane].x;
            beta[(int64_t)c * mmax + jc] = b;
        }
    }
}

// Ritz value after step jv[c]; on convergence (or at the step cap) the slot
// is marked finished (active = 2), otherwise its step advances.
// The tridiagonal work runs in the precision of the recurrence: FP32 in mixed
// mode (the returned sigma there comes from the refined Rayleigh quotient, the
// Ritz value only steers), FP64 otherwise.
template <typename real>
__global__ void slot_tridiag_kernel(int S, int mmax, const double *__restrict__ alpha, const double *__restrict__ beta,
                                    int *__restrict__ active, int *__restrict__ jv, double *__restrict__ theta,
                                    double *__restrict__ svec, int *__restrict__ convd, double tol_q,
                                    double tol_floor) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= S || active[c] != 1) return;
    const int j = jv[c], k = j + 1;
    real a[LANCZOS_MMAX], b[LANCZOS_MMAX], s[LANCZOS_MMAX], wk[5 * LANCZOS_MMAX];
    for (int i = 0; i < k; ++i) { a[i] = (real)alpha[(int64_t)c * mmax + i]; b[i] = (real)beta[(int64_t)c * mmax + i]; }
    const real th1 = tridiag_eig<real>(a, b, k, k - 1);
    const real th2 = k > 1 ? tridiag_eig<real>(a, b, k, k - 2) : (real)0;
    tridiag_vec<real>(a, b, k, th1, s, wk);
    const double rb = fabs((double)b[k - 1] * (double)s[k - 1]);
    const double gap = fmax((double)th1 - (double)th2, 1e-300);
    const double est = rb * rb / ((double)th1 * gap);
    const bool breakdown = (double)b[k - 1] <= 1e-300 * (double)th1;
    const bool conv = breakdown || est <= tol_q || rb <= tol_floor * (double)th1;
    theta[c] = (double)th1;
    for (int i = 0; i < k; ++i) svec[(int64_t)c * mmax + i] = (double)s[i];
    if (conv || k == mmax) {
        active[c] = 2;
        convd[c] = conv ? 1 : 0;
    } else {
        jv[c] = j + 1;
    }
}

// Bookkeeping of the harvest, one thread per slot: a converged slot (state 2)
// gets its place in the finished buffer and is listed for its Ritz vector; a
// converged or empty slot (state 3) takes the next point and is listed for the
// refill of its start vector.
__global__ void slot_book_kernel(int S, int *__restrict__ jv, int *__restrict__ active,
                                 const double *__restrict__ theta, const int *__restrict__ convd, int *__restrict__ pt,
                                 double2 *__restrict__ zslot, const double2 *__restrict__ zall, int npts,
                                 int *__restrict__ counters, int *__restrict__ fin_pt, double2 *__restrict__ fin_z,
                                 double *__restrict__ fin_theta, int *__restrict__ fin_conv, int4 *__restrict__ work) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= S) return;
    const int st = active[c];
    if (st == 2) {
        const int dest = atomicAdd(&counters[1], 1);
        fin_pt[dest] = pt[c];
        fin_z[dest] = zslot[c];
        fin_theta[dest] = theta[c];
        fin_conv[dest] = convd[c];
        work[atomicAdd(&counters[2], 1)] = make_int4(c, dest, jv[c] + 1, 0);
    }
    if (st == 2 || st == 3) {
        const int nxt = atomicAdd(&counters[0], 1);
        if (nxt < npts) {
            pt[c] = nxt;
            zslot[c] = zall[nxt];
            jv[c] = 0;
            active[c] = 1;
            work[S + atomicAdd(&counters[3], 1)] = make_int4(c, 0, 0, 0);
        } else {
            active[c] = 0;
        }
    }
}

// Ritz vectors of the listed slots: U[:, dest] = Q_{0:k} svec, one thread per
// (slot, row); the basis of a slot is strided by S, so this is a gather with
// many independent loads in flight.
template <typename real>
__global__ void __launch_bounds__(256)
slot_ritz_kernel(const cx_t<real> *__restrict__ Q, int64_t qs, int n, int S, int mmax, const double *__restrict__ svec,
                 const int4 *__restrict__ work, const int *__restrict__ cnt, double2 *__restrict__ Ufin, int F) {
    const int64_t total = (int64_t)(*cnt) * n;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
        const int4 e = work[w / n];
        const int i = (int)(w % n), c = e.x, k = e.z;
        const cx_t<real> *q = Q + (int64_t)i * S + c;
        const double *sv = svec + (int64_t)c * mmax;
        real ur = 0, ui = 0, vr = 0, vi = 0;
        int t = 0;
        for (; t + 1 < k; t += 2) {
            const cx_t<real> a = q[(int64_t)t * qs], b = q[(int64_t)(t + 1) * qs];
            const real sa = (real)sv[t], sb = (real)sv[t + 1];
            ur += sa * a.x; ui += sa * a.y;
            vr += sb * b.x; vi += sb * b.y;
        }
        if (t < k) {
            const cx_t<real> a = q[(int64_t)t * qs];
            const real sa = (real)sv[t];
            ur += sa * a.x; ui += sa * a.y;
        }
        Ufin[(int64_t)i * F + e.y] = make_double2((double)(ur + vr), (double)(ui + vi));
    }
}

// Start vectors of the refilled slots: the common seeded vector v0, or, when
// vw is given, the point's own unit start vector, column posw[offw + pt] (or
// offw + pt) of the row-major n x ldw array vw.
template <typename real>
__global__ void __launch_bounds__(256)
slot_refill_kernel(cx_t<real> *__restrict__ Q, int n, int S, const int4 *__restrict__ work, const int *__restrict__ cnt,
                   const double2 *__restrict__ v0, const int *__restrict__ pt, const double2 *__restrict__ vw,
                   int64_t ldw, const int *__restrict__ posw, int offw) {
    const int64_t total = (int64_t)(*cnt) * n;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
        const int c = work[w / n].x, i = (int)(w % n);
        double2 v;
        if (vw) {
            const int k = offw + pt[c];
            v = vw[(int64_t)i * ldw + (posw ? posw[k] : k)];
        } else {
            v = v0[i];
        }
        Q[(int64_t)i * S + c] = mk<real>((real)v.x, (real)v.y);
    }
}

// Results of finished points t < P (sigma from theta or from the Rayleigh
// quotient s2), scattered to their grid positions.
__global__ void fin_scatter_kernel(int P_host, const int *__restrict__ P_dev, const int *__restrict__ fin_pt, const double2 *__restrict__ fin_z,
                                   const double *__restrict__ fin_theta, const int *__restrict__ fin_conv,
                                   const double *__restrict__ s2, const double *__restrict__ rr, int use_rq,
                                   double norm2, const double *__restrict__ eps, int neps, double *__restrict__ sigma_out,
                                   double *__restrict__ res_out, int32_t *__restrict__ flags_out,
                                   uint32_t *__restrict__ member_out, int *__restrict__ nbad, double u_solve,
                                   double fb_ku, int *__restrict__ fb_list, int *__restrict__ fb_cnt,
                                   const double2 *__restrict__ U0, int64_t ldu, double2 *__restrict__ warm,
                                   int64_t ldw, int n, const double2 *__restrict__ v0) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int P = P_dev ? min(*P_dev, P_host) : P_host;
    if (t >= P) return;
    const double th = fin_theta[t];
    const double rq = sqrt(fmax(s2[t], 0.0));
    const double sl = th > 0.0 ? 1.0 / sqrt(th) : 0.0;
    const double sig = use_rq ? rq : sl;
    const double2 z = fin_z[t];
    const double mz = norm2 + sqrt(z.x * z.x + z.y * z.y);
    const int g = fin_pt[t];
    if (fb_list) {
        // mixed precision cannot be trusted here: the FP32 recurrence did not
        // converge, or kappa = ||M|| / sigma is so large that the refinement
        // of the solves stops contracting; such points are redone in FP64
        const double sg = fmin(sig, sl > 0.0 ? sl : sig);
        if (!fin_conv[t] || !(sg > 0.0) || (mz / sg) * u_solve > fb_ku) {
            const int k = atomicAdd(fb_cnt, 1);
            fb_list[k] = g;
            // the point's (unit) Ritz vector starts its FP64 recurrence; a point
            // whose FP32 recurrence broke down starts from the common vector v0
            if (warm) {
                const bool good = isfinite(th) && th > 0.0;
                for (int i = 0; i < n; ++i) warm[(int64_t)i * ldw + k] = good ? U0[(int64_t)i * ldu + t] : v0[i];
            }
            return;
        }
    }
    int fl = PSEUDO_PT_REFINED;
    if (!fin_conv[t]) { fl |= PSEUDO_PT_NOT_CONVERGED; atomicAdd(nbad, 1); }
    sigma_out[g] = sig;
    if (res_out) res_out[g] = rq > 0.0 ? rr[t] / (rq * mz) : 0.0;
    if (flags_out) flags_out[g] = fl;
    if (member_out) {
        uint32_t m = 0;
        for (int e = 0; e < neps; ++e) m |= (sig < eps[e] ? 1u : 0u) << e;
        member_out[g] = m;
    }
}

template <typename real>
void launch_slot_copy(const cx_t<real> *Q, int64_t qs, cx_t<real> *W, int n, int S, const int *jv, const int *active,
                      cudaStream_t s) {
    note_launch(); slot_copy_kernel<real><<<(S + 31) / 32, 256, 0, s>>>(Q, qs, W, n, S, jv, active);
}
template <typename real>
void launch_slot_orth(cx_t<real> *Q, int64_t qs, cx_t<real> *W, int n, int S, const int *jv, int mmax,
                      const int *active, double *alpha, double *beta, int passes, cudaStream_t s) {
    note_launch(); slot_orth_kernel<real><<<(S + 31) / 32, ORTH_WARPS * 32, 0, s>>>(Q, qs, W, n, S, jv, mmax, active, alpha, beta,
                                                                                 passes);
}
void launch_slot_tridiag(int S, int mmax, const double *alpha, const double *beta, int *active, int *jv, double *theta,
                         double *svec, int *convd, double tol_q, double tol_floor, int fp32, cudaStream_t s) {
    note_launch();
    if (fp32)
        slot_tridiag_kernel<float><<<(S + 63) / 64, 64, 0, s>>>(S, mmax, alpha, beta, active, jv, theta, svec, convd,
                                                               tol_q, tol_floor);
    else
        slot_tridiag_kernel<double><<<(S + 63) / 64, 64, 0, s>>>(S, mmax, alpha, beta, active, jv, theta, svec, convd,
                                                                tol_q, tol_floor);
}
template <typename real>
void launch_slot_harvest(cx_t<real> *Q, int64_t qs, int n, int S, int mmax, const double *svec, int *jv, int *active,
                         const double *theta, const int *convd, int *pt, double2 *zslot, const double2 *zall, int npts,
                         int *counters, double2 *Ufin, int F, int *fin_pt, double2 *fin_z, double *fin_theta,
                         int *fin_conv, const double2 *v0, int4 *work, cudaStream_t s, const double2 *vw,
                         int64_t ldw, const int *posw, int offw) {
    cudaMemsetAsync(counters + 2, 0, 2 * sizeof(int), s);
    note_launch();
    slot_book_kernel<<<(S + 255) / 256, 256, 0, s>>>(S, jv, active, theta, convd, pt, zslot, zall, npts, counters,
                                                     fin_pt, fin_z, fin_theta, fin_conv, work);
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    note_launch();
    slot_ritz_kernel<real><<<nsm * 8, 256, 0, s>>>(Q, qs, n, S, mmax, svec, work, counters + 2, Ufin, F);
    note_launch();
    slot_refill_kernel<real><<<nsm * 8, 256, 0, s>>>(Q, n, S, work + S, counters + 3, v0, pt, vw, ldw, posw, offw);
}
void launch_fin_scatter(int P, const int *fin_pt, const double2 *fin_z, const double *fin_theta, const int *fin_conv,
                        const double *s2, const double *rr, int use_rq, double norm2, const double *eps, int neps,
                        double *sigma_out, double *res_out, int32_t *flags_out, uint32_t *member_out, int *nbad,
                        double u_solve, double fb_ku, int *fb_list, int *fb_cnt, cudaStream_t s, const double2 *U0,
                        int64_t ldu, double2 *warm, int64_t ldw, int n, const double2 *v0, const int *P_dev) {
    if (P > 0) {
        note_launch(); fin_scatter_kernel<<<(P + 127) / 128, 128, 0, s>>>(P, P_dev, fin_pt, fin_z, fin_theta, fin_conv, s2, rr, use_rq, norm2,
                                                                        eps, neps, sigma_out, res_out, flags_out,
                                                                        member_out, nbad, u_solve, fb_ku, fb_list,
                                                                        fb_cnt, U0, ldu, warm, ldw, n, v0);
    }
}

// mask[c] = 1 for c < *P, 0 for the other columns up to F
__global__ void mask_prefix_kernel(int *__restrict__ mask, int F, const int *__restrict__ P) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < F) mask[c] = c < *P ? 1 : 0;
}
void launch_mask_prefix(int *mask, int F, const int *P, cudaStream_t s) {
    if (F > 0) { note_launch(); mask_prefix_kernel<<<(F + 255) / 256, 256, 0, s>>>(mask, F, P); }
}

// Loop control of the device-driven Lanczos driver (one thread), after the
// compaction of the running slots: finish the finished buffer when it holds
// S points or when no slot runs and it is not empty; step while a slot runs.
// The loop stops early after `guard` iterations of one launch, or when a
// bounded wait of a tensor-core kernel gave up (err[0]); the host then
// resumes or reports.  ctl[0] counts this launch's iterations (zeroed by the
// launch), stat[0] the steps, stat[1] the solves (2 per running slot and
// step), stat[2] the Rayleigh-quotient products of the finishes (2 per
// point), stat[3] the finishes.  With graph = 0 it only counts.
__global__ void lanc_ctrl_kernel(const int *__restrict__ cnt, const int *__restrict__ counters, int S,
                                 const int *__restrict__ err, long long guard, long long *__restrict__ ctl,
                                 long long *__restrict__ stat, cudaGraphConditionalHandle hw,
                                 cudaGraphConditionalHandle hf, cudaGraphConditionalHandle hs, int graph) {
    if (threadIdx.x | blockIdx.x) return;
    const int c = *cnt, nfin = counters[1];
    const long long it = ++ctl[0];
    const bool fin = nfin >= S || (c == 0 && nfin > 0);
    const bool ok = err[0] == 0;
    const bool step = c > 0 && ok;
    if (fin && ok) { stat[2] += 2 * (long long)nfin; stat[3] += 1; }
    if (step) { stat[0] += 1; stat[1] += 2 * (long long)c; }
    if (graph) {
        cudaGraphSetConditional(hf, fin && ok ? 1u : 0u);
        cudaGraphSetConditional(hs, step ? 1u : 0u);
        cudaGraphSetConditional(hw, step && it < guard ? 1u : 0u);
    }
}
void launch_lanc_ctrl(const int *cnt, const int *counters, int S, const int *err, long long guard, long long *ctl,
                      long long *stat, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hf,
                      cudaGraphConditionalHandle hs, int graph, cudaStream_t s) {
    note_launch();
    lanc_ctrl_kernel<<<1, 32, 0, s>>>(cnt, counters, S, err, guard, ctl, stat, hw, hf, hs, graph);
}

__global__ void fb_gather_kernel(const int *__restrict__ list, int cnt, const double2 *__restrict__ zall,
                                 double2 *__restrict__ zc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) zc[t] = zall[list[t]];
}
__global__ void fb_scatter_kernel(const int *__restrict__ list, int cnt, const double *__restrict__ sc,
                                  const double *__restrict__ rc, const int32_t *__restrict__ fc,
                                  const uint32_t *__restrict__ mc, double *__restrict__ sigma, double *__restrict__ res,
                                  int32_t *__restrict__ flags, uint32_t *__restrict__ member) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int g = list[t];
    sigma[g] = sc[t];
    if (res) res[g] = rc[t];
    if (flags) flags[g] = fc[t] | PSEUDO_PT_IR_FALLBACK;
    if (member) member[g] = mc[t];
}
void launch_fb_gather(const int *list, int cnt, const double2 *zall, double2 *zc, cudaStream_t s) {
    if (cnt > 0) { note_launch(); fb_gather_kernel<<<(cnt + 127) / 128, 128, 0, s>>>(list, cnt, zall, zc); }
}
void launch_fb_scatter(const int *list, int cnt, const double *sc, const double *rc, const int32_t *fc,
                       const uint32_t *mc, double *sigma, double *res, int32_t *flags, uint32_t *member,
                       cudaStream_t s) {
    if (cnt > 0) {
        note_launch();
        fb_scatter_kernel<<<(cnt + 127) / 128, 128, 0, s>>>(list, cnt, sc, rc, fc, mc, sigma, res, flags, member);
    }
}
template void launch_slot_copy<float>(const float2 *, int64_t, float2 *, int, int, const int *, const int *, cudaStream_t);
template void launch_slot_copy<double>(const double2 *, int64_t, double2 *, int, int, const int *, const int *, cudaStream_t);
template void launch_slot_orth<float>(float2 *, int64_t, float2 *, int, int, const int *, int, const int *, double *,
                                      double *, int, cudaStream_t);
template void launch_slot_orth<double>(double2 *, int64_t, double2 *, int, int, const int *, int, const int *, double *,
                                       double *, int, cudaStream_t);
template void launch_slot_harvest<float>(float2 *, int64_t, int, int, int, const double *, int *, int *, const double *,
                                         const int *, int *, double2 *, const double2 *, int, int *, double2 *, int,
                                         int *, double2 *, double *, int *, const double2 *, int4 *, cudaStream_t,
                                         const double2 *, int64_t, const int *, int);
template void launch_slot_harvest<double>(double2 *, int64_t, int, int, int, const double *, int *, int *,
                                          const double *, const int *, int *, double2 *, const double2 *, int, int *,
                                          double2 *, int, int *, double2 *, double *, int *, const double2 *, int4 *,
                                          cudaStream_t, const double2 *, int64_t, const int *, int);

}  // namespace pseudo

// ============ grid-parallel reorthogonalisation for the slot scheme
// One classical Gram-Schmidt pass is split into a dot kernel and an update
// kernel whose CTAs each own 32 columns x a slice of rows, so that the whole
// GPU streams Q (the pass is bound by reading Q twice).
namespace pseudo {
constexpr int OS_ROWS = 128;  // rows per CTA slice

template <typename real>
__global__ void __launch_bounds__(ORTH_WARPS * 32)
orth_dots_kernel(const cx_t<real> *__restrict__ Q, int64_t qs, const cx_t<real> *__restrict__ W, int n, int S,
                 const int *__restrict__ jv, const int *__restrict__ active, int ldh, double2 *__restrict__ Hp) {
    using C = cx_t<real>;
    __shared__ double2 red[ORTH_WARPS][TCH][32];
    __shared__ int s_jmax;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const bool on = (c < S) && active[c] == 1;
    const int jc = on ? jv[c] : -1;
    if (threadIdx.x == 0) s_jmax = -1;
    __syncthreads();
    if (warp == 0 && on) atomicMax(&s_jmax, jc);
    __syncthreads();
    const int jmax = s_jmax;
    if (jmax < 0) return;
    const int r0 = blockIdx.y * OS_ROWS, r1 = min(n, r0 + OS_ROWS);
    const int cc = on ? c : 0;
    for (int t0 = 0; t0 <= jmax; t0 += TCH) {
        C acc[TCH];
#pragma unroll
        for (int u = 0; u < TCH; ++u) acc[u] = mk<real>(0, 0);
        if (on && t0 <= jc)
            for (int i = r0 + warp; i < r1; i += ORTH_WARPS) {
                const C wv = W[(int64_t)i * S + cc];
#pragma unroll
                for (int u = 0; u < TCH; ++u)
                    if (t0 + u <= jc) cfma(acc[u], cconj(Q[(int64_t)(t0 + u) * qs + (int64_t)i * S + cc]), wv);
            }
#pragma unroll
        for (int u = 0; u < TCH; ++u) red[warp][u][lane] = make_double2((double)acc[u].x, (double)acc[u].y);
        __syncthreads();
        for (int e = threadIdx.x; e < TCH * 32; e += blockDim.x) {
            const int u = e / 32, l = e % 32, col = blockIdx.x * 32 + l;
            if (col < S && active[col] == 1 && t0 + u <= jv[col]) {
                double2 s = make_double2(0.0, 0.0);
                for (int w = 0; w < ORTH_WARPS; ++w) { s.x += red[w][u][l].x; s.y += red[w][u][l].y; }
                atomicAdd(&Hp[(int64_t)col * ldh + t0 + u].x, s.x);
                atomicAdd(&Hp[(int64_t)col * ldh + t0 + u].y, s.y);
            }
        }
        __syncthreads();
    }
}

// w -= sum_t h_t q_t over the slice's rows; partial ||w||^2 into nrm2 (when
// non-null) and, from the first slice, alpha_acc += Re h_{j}.
template <typename real>
__global__ void __launch_bounds__(ORTH_WARPS * 32)
orth_update_kernel(const cx_t<real> *__restrict__ Q, int64_t qs, cx_t<real> *__restrict__ W, int n, int S,
                   const int *__restrict__ jv, const int *__restrict__ active, int ldh, const double2 *__restrict__ Hp,
                   double *__restrict__ nrm2, double *__restrict__ alpha_acc) {
    using C = cx_t<real>;
    __shared__ double s_n[ORTH_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const bool on = (c < S) && active[c] == 1;
    const int jc = on ? jv[c] : -1;
    const int r0 = blockIdx.y * OS_ROWS, r1 = min(n, r0 + OS_ROWS);
    const int cc = on ? c : 0;
    real sp = 0;
    if (on) {
        if (blockIdx.y == 0 && warp == 0) alpha_acc[c] += Hp[(int64_t)c * ldh + jc].x;
        for (int t0 = 0; t0 <= jc; t0 += TCH) {
            C hc[TCH];
#pragma unroll
            for (int u = 0; u < TCH; ++u) {
                const double2 hv = t0 + u <= jc ? Hp[(int64_t)c * ldh + t0 + u] : make_double2(0.0, 0.0);
                hc[u] = mk<real>((real)hv.x, (real)hv.y);
            }
            const bool last = t0 + TCH > jc;
            for (int i = r0 + warp; i < r1; i += ORTH_WARPS) {
                C wv = W[(int64_t)i * S + cc];
#pragma unroll
                for (int u = 0; u < TCH; ++u)
                    if (t0 + u <= jc) cfms(wv, Q[(int64_t)(t0 + u) * qs + (int64_t)i * S + cc], hc[u]);
                W[(int64_t)i * S + cc] = wv;
                if (last) sp += wv.x * wv.x + wv.y * wv.y;
            }
        }
    }
    if (!nrm2) return;
    s_n[warp][lane] = (double)sp;
    __syncthreads();
    if (warp == 0 && on) {
        double t = 0.0;
        for (int w = 0; w < ORTH_WARPS; ++w) t += s_n[w][lane];
        atomicAdd(&nrm2[c], t);
    }
}

// q_{j+1} = w / ||w||, alpha_j, beta_j
template <typename real>
__global__ void __launch_bounds__(ORTH_WARPS * 32)
orth_finish_kernel(cx_t<real> *__restrict__ Q, int64_t qs, const cx_t<real> *__restrict__ W, int n, int S,
                   const int *__restrict__ jv, const int *__restrict__ active, const double *__restrict__ nrm2,
                   const double *__restrict__ alpha_acc, int mmax, double *__restrict__ alpha,
                   double *__restrict__ beta) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    if (c >= S || active[c] != 1) return;
    const int jc = jv[c];
    const double b = sqrt(nrm2[c]);
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    const int r0 = blockIdx.y * OS_ROWS, r1 = min(n, r0 + OS_ROWS);
    for (int i = r0 + warp; i < r1; i += ORTH_WARPS) {
        const cx_t<real> wv = W[(int64_t)i * S + c];
        Q[(int64_t)(jc + 1) * qs + (int64_t)i * S + c] = mk<real>((real)(wv.x * inv), (real)(wv.y * inv));
    }
    if (blockIdx.y == 0 && warp == 0) {
        alpha[(int64_t)c * mmax + jc] = alpha_acc[c];
        beta[(int64_t)c * mmax + jc] = b;
    }
}

template <typename real>
void launch_slot_orth_grid(cx_t<real> *Q, int64_t qs, cx_t<real> *W, int n, int S, const int *jv, int mmax,
                           const int *active, double *alpha, double *beta, int passes, double2 *Hp, double *nrm2,
                           double *alpha_acc, cudaStream_t s) {
    const dim3 grid((S + 31) / 32, (n + OS_ROWS - 1) / OS_ROWS);
    const int ldh = mmax + 1;
    cudaMemsetAsync(alpha_acc, 0, sizeof(double) * S, s);
    cudaMemsetAsync(nrm2, 0, sizeof(double) * S, s);
    for (int pass = 0; pass < passes; ++pass) {
        cudaMemsetAsync(Hp, 0, sizeof(double2) * (size_t)S * ldh, s);
        note_launch(); orth_dots_kernel<real><<<grid, ORTH_WARPS * 32, 0, s>>>(Q, qs, W, n, S, jv, active, ldh, Hp);
        note_launch(); orth_update_kernel<real><<<grid, ORTH_WARPS * 32, 0, s>>>(Q, qs, W, n, S, jv, active, ldh, Hp,
                                                                                 pass == passes - 1 ? nrm2 : nullptr,
                                                                                 alpha_acc);
    }
    note_launch(); orth_finish_kernel<real><<<grid, ORTH_WARPS * 32, 0, s>>>(Q, qs, W, n, S, jv, active, nrm2, alpha_acc,
                                                                             mmax, alpha, beta);
}
template void launch_slot_orth_grid<float>(float2 *, int64_t, float2 *, int, int, const int *, int, const int *, double *,
                                           double *, int, double2 *, double *, double *, cudaStream_t);
template void launch_slot_orth_grid<double>(double2 *, int64_t, double2 *, int, int, const int *, int, const int *,
                                            double *, double *, int, double2 *, double *, double *, cudaStream_t);
}  // namespace pseudo
