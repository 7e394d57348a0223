// Fast Rayleigh--Ritz-SVD on the recycled subspace (Alg. 1, recySing), one
// CTA per grid point, all in FP64.  For the lane's basis V (n x k, k = p r)
// with W1 = T V, W3 = T^H T V, W4 = T^H V and the projected Grams
// H1 = W1^H W1, H2 = W1^H V (eq. (H) with M = T, S = I, so H3 = I,
// W2 = W6 = V and W5 = W1):
//   1. H(z) = H1 - z H2 - conj(z) H2^H + (|z|^2 + eps) I      (eq. (rayleighN))
//      and its eigenpairs (Theta ascending, G)                  (eq. (step1))
//   2. r~ = smallest j >= r with theta_{j+1} - theta_j > theta_k eps_m / tau
//      (eq. (tau)), then capped at RTMAX columns: the Ritz pairs come from
//      the span of V G_{1:min(r~, RTMAX)}, a subspace of span V, so they stay
//      upper bounds and the acceptance test below judges the pair actually
//      returned; the cap can only cost acceptances.  rt_out gets the
//      uncapped r~.
//   3. Y = (W1 - z V) G_{1:r~}; R~ from the Gram Y^H Y by a column-scaled
//      Cholesky (Y's columns are orthogonal up to rounding, so the scaled
//      Gram is close to I and the factor keeps full relative accuracy);
//      one-sided Jacobi SVD of R~ -> xi~ (ascending), G~          (eq. (step2))
//   4. w_j = (W3 - z W4 - conj(z) W1 + (|z|^2 - xi_j^2) V) c_j with
//      c_j = G_{1:r~} G~_{:,j}, j = 1, 2 (eq. (fastresidual))
//   5. accept iff ||w_1|| <= max(eta xi_1 ||M(z)||, ||M(z)||^2 eps_m)
//      (eq. (tolC)) and, when rtol > 0, the Kato--Temple estimate
//      ||w_1||^2 / (2 xi_1^2 (xi_2^2 - xi_1^2 - ||w_2||)) <= rtol / 4.
// For rejected points the coefficients C_X = G_{1:r~} G~_{:,1:r} of the Ritz
// vectors X~ = V C_X are written out as the warm start of the refinement.
#include "common.cuh"
#include "internal.h"
#include "recycle.h"
#include "smalldense.cuh"

namespace pseudo {

constexpr int RS_THREADS = 256;
constexpr int RS_CH = 32;  // rows per chunk when forming Y

struct RecySingArgs {
    int n, KM, r, npts;
    int64_t ldv;                      // row stride of the lane arrays
    const double2 *V, *W1, *W3, *W4;  // lane l's block starts at + l * KM
    const double2 *H1, *H2;           // lane l at + l * KM * KM
    const int *p;                     // blocks per lane
    const double2 *z;                 // per point
    const int *lane;                  // per point
    double eps_shift, tau, eta, rtol, norm2;
    double *sigma, *res, *xi2, *w2;
    int *accept, *rt;
    double2 *CX;                      // per point KM x r (row-major, ld r)
};

__global__ void __launch_bounds__(RS_THREADS) recysing_kernel(RecySingArgs a) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int j = blockIdx.x;
    if (j >= a.npts) return;
    const int tid = threadIdx.x;
    const int l = a.lane[j];
    const int k = a.p[l] * a.r;
    const int KM = a.KM;
    const double2 z = a.z[j];
    const double zz = z.x * z.x + z.y * z.y;
    const double Mz = a.norm2 + sqrt(zz);
    if (k == 0) {
        if (tid == 0) {
            a.sigma[j] = 0.0; a.res[j] = 1.0; a.accept[j] = 0; a.rt[j] = 0; a.xi2[j] = 0.0; a.w2[j] = 0.0;
        }
        return;
    }
    double2 *H = (double2 *)sm_raw;       // k x k
    double2 *G = H + KM * KM;             // k x k
    double2 *Gr = G + KM * KM;            // k x RTMAX
    double2 *Yc = Gr + KM * RTMAX;        // RS_CH x RTMAX
    double2 *Rt = Yc + RS_CH * RTMAX;     // RTMAX x RTMAX
    double2 *Vr = Rt + RTMAX * RTMAX;     // RTMAX x RTMAX
    double2 *cc = Vr + RTMAX * RTMAX;     // k x 2 (c_1, c_2)
    double *theta = (double *)(cc + 2 * KM);
    double *rot = theta + KM;             // 224 doubles
    double *sig = rot + 224;              // RTMAX
    int *perm = (int *)(sig + RTMAX);     // KM
    __shared__ int s_rt, s_ok, s_rt_rule;
    __shared__ double s_w[2][RS_THREADS / 32];

    const int64_t ldv = a.ldv;
    const double2 *V = a.V + (int64_t)l * KM, *W1 = a.W1 + (int64_t)l * KM;
    const double2 *W3 = a.W3 + (int64_t)l * KM, *W4 = a.W4 + (int64_t)l * KM;
    const double2 *H1 = a.H1 + (int64_t)l * KM * KM, *H2 = a.H2 + (int64_t)l * KM * KM;

    // 1. H(z)
    for (int e = tid; e < k * k; e += RS_THREADS) {
        const int p = e / k, q = e % k;
        double2 h = H1[p * KM + q];
        const double2 a2 = H2[p * KM + q];
        const double2 b2 = cconj(H2[q * KM + p]);  // (H2^H)_{pq}
        cfms(h, z, a2);
        cfms(h, cconj(z), b2);
        if (p == q) { h.x += zz + a.eps_shift; h.y = 0.0; }
        H[e] = h;
    }
    __syncthreads();
    blk_heev_jacobi(H, G, k, rot);
    blk_sort_diag(H, k, perm, theta);
    // 2. r~ (eq. (tau)), 1-based j in [r, k-1]
    if (tid == 0) {
        int rt = k;
        const double thr = theta[k - 1] * 2.220446049250313e-16 / a.tau;
        for (int jj = a.r; jj < k; ++jj)
            if (fabs(theta[jj - 1] - theta[jj]) > thr) { rt = jj; break; }
        s_rt_rule = rt;  // reported: r~ of eq. (tau) before the cap
        if (rt > RTMAX) rt = RTMAX;
        if (rt > k) rt = k;
        s_rt = rt;
        s_ok = 1;
    }
    __syncthreads();
    const int rt = s_rt;
    for (int e = tid; e < k * rt; e += RS_THREADS) {
        const int t = e / rt, c = e % rt;
        Gr[t * RTMAX + c] = G[t * k + perm[c]];
    }
    __syncthreads();
    // 3. Gram of Y = (W1 - zV) Gr, Y formed a chunk of rows at a time
    double2 gacc = make_double2(0.0, 0.0);
    const int ga = tid / RTMAX, gb = tid % RTMAX;
    for (int r0 = 0; r0 < a.n; r0 += RS_CH) {
        const int rows = min(RS_CH, a.n - r0);
        for (int e = tid; e < rows * rt; e += RS_THREADS) {
            const int i = e / rt, c = e % rt;
            const double2 *w1r = W1 + (int64_t)(r0 + i) * ldv, *vr = V + (int64_t)(r0 + i) * ldv;
            double2 acc = make_double2(0.0, 0.0);
            for (int t = 0; t < k; ++t) {
                double2 u = w1r[t];
                cfms(u, z, vr[t]);
                cfma(acc, u, Gr[t * RTMAX + c]);
            }
            Yc[i * RTMAX + c] = acc;
        }
        __syncthreads();
        if (ga < rt && gb < rt)
            for (int i = 0; i < rows; ++i) cfma(gacc, cconj(Yc[i * RTMAX + ga]), Yc[i * RTMAX + gb]);
        __syncthreads();
    }
    // column-scaled Cholesky of the Gram -> R~ (rt x rt, stored with ld rt)
    __shared__ double s_d[RTMAX];
    if (ga < rt && gb < rt) Rt[ga * rt + gb] = gacc;
    __syncthreads();
    if (tid < rt) s_d[tid] = sqrt(fmax(Rt[tid * rt + tid].x, 0.0));
    __syncthreads();
    if (ga < rt && gb < rt) {
        const double d = s_d[ga] * s_d[gb];
        Rt[ga * rt + gb] = d > 0.0 ? cscale(Rt[ga * rt + gb], 1.0 / d) : make_double2(ga == gb ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    const bool okc = blk_cholesky(Rt, rt);
    if (ga < rt && gb < rt) Rt[ga * rt + gb] = cscale(Rt[ga * rt + gb], s_d[gb]);
    __syncthreads();
    // SVD of R~
    blk_svd_jacobi(Rt, Vr, rt, rot);
    blk_colnorms(Rt, rt, sig);
    if (tid == 0) {
        // ascending order of the singular values
        for (int q = 0; q < rt; ++q) perm[q] = q;
        for (int q = 1; q < rt; ++q) {
            int x = perm[q];
            int w = q - 1;
            while (w >= 0 && sig[perm[w]] > sig[x]) { perm[w + 1] = perm[w]; --w; }
            perm[w + 1] = x;
        }
        if (!okc) s_ok = 0;
    }
    __syncthreads();
    const double xi1 = sig[perm[0]];
    const double xi2v = rt > 1 ? sig[perm[1]] : 0.0;
    // coefficient vectors c_j = Gr G~_{:,j} (j = 1..r written as C_X; j = 1,2 kept)
    const int nr = min(a.r, rt);
    double2 *CXj = a.CX + (int64_t)j * KM * a.r;
    for (int e = tid; e < k * a.r; e += RS_THREADS) {
        const int t = e / a.r, c = e % a.r;
        double2 acc = make_double2(0.0, 0.0);
        if (c < nr) {
            const int pc = perm[c];
            for (int q = 0; q < rt; ++q) cfma(acc, Gr[t * RTMAX + q], Vr[q * rt + pc]);
        }
        CXj[t * a.r + c] = acc;
        if (c < 2) cc[t * 2 + c] = acc;
    }
    for (int e = k * a.r + tid; e < KM * a.r; e += RS_THREADS) CXj[e] = make_double2(0.0, 0.0);
    __syncthreads();
    // 4. residual norms ||w_1||, ||w_2|| (eq. (fastresidual))
    const double2 zc = cconj(z);
    double s1 = 0.0, s2 = 0.0;
    const double d1 = zz - xi1 * xi1, d2 = zz - xi2v * xi2v;
    for (int i = tid; i < a.n; i += RS_THREADS) {
        const double2 *w3 = W3 + (int64_t)i * ldv, *w4 = W4 + (int64_t)i * ldv, *w1 = W1 + (int64_t)i * ldv,
                      *v = V + (int64_t)i * ldv;
        double2 u1 = make_double2(0.0, 0.0), u2 = u1;
        for (int t = 0; t < k; ++t) {
            double2 base = w3[t];
            cfms(base, z, w4[t]);
            cfms(base, zc, w1[t]);
            const double2 vt = v[t];
            double2 e1 = base, e2 = base;
            e1.x += d1 * vt.x; e1.y += d1 * vt.y;
            e2.x += d2 * vt.x; e2.y += d2 * vt.y;
            cfma(u1, e1, cc[t * 2]);
            cfma(u2, e2, cc[t * 2 + 1]);
        }
        s1 += cabs2(u1);
        s2 += cabs2(u2);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((tid & 31) == 0) { s_w[0][tid >> 5] = s1; s_w[1][tid >> 5] = s2; }
    __syncthreads();
    if (tid == 0) {
        double a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < RS_THREADS / 32; ++w) { a1 += s_w[0][w]; a2 += s_w[1][w]; }
        const double nw1 = sqrt(a1), nw2 = sqrt(a2);
        // 5. acceptance (eq. (tolC)) and the accuracy estimate
        bool acc = s_ok && xi1 > 0.0 && nw1 <= fmax(a.eta * xi1 * Mz, Mz * Mz * 2.220446049250313e-16);
        if (acc && a.rtol > 0.0) {
            if (rt < 2) acc = false;
            else {
                const double gap = xi2v * xi2v - xi1 * xi1 - nw2;
                const double est = gap > 0.0 ? nw1 * nw1 / (2.0 * xi1 * xi1 * gap) : 1e300;
                acc = est <= a.rtol / 4.0;
            }
        }
        a.sigma[j] = xi1;
        a.res[j] = xi1 > 0.0 ? nw1 / (xi1 * Mz) : 1e300;
        a.accept[j] = acc ? 1 : 0;
        a.rt[j] = s_rt_rule;
        a.xi2[j] = xi2v;
        a.w2[j] = nw2;
    }
}

size_t recysing_smem(int KM) {
    return sizeof(double2) * (size_t)(2 * KM * KM + KM * RTMAX + RS_CH * RTMAX + 2 * RTMAX * RTMAX + 2 * KM) +
           sizeof(double) * (size_t)(KM + 224 + RTMAX) + sizeof(int) * KM + 64;
}

cudaError_t launch_recysing(const RecySingLaunch &L, cudaStream_t s) {
    if (L.npts <= 0) return cudaSuccess;
    RecySingArgs a;
    a.n = L.n; a.KM = L.KM; a.r = L.r; a.npts = L.npts; a.ldv = L.ldv;
    a.V = L.V; a.W1 = L.W1; a.W3 = L.W3; a.W4 = L.W4; a.H1 = L.H1; a.H2 = L.H2; a.p = L.p;
    a.z = L.z; a.lane = L.lane;
    a.eps_shift = L.eps_shift; a.tau = L.tau; a.eta = L.eta; a.rtol = L.rtol; a.norm2 = L.norm2;
    a.sigma = L.sigma; a.res = L.res; a.xi2 = L.xi2; a.w2 = L.w2; a.accept = L.accept; a.rt = L.rt; a.CX = L.CX;
    const size_t sm = recysing_smem(L.KM);
    cudaFuncSetAttribute(recysing_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    note_launch(); recysing_kernel<<<L.npts, RS_THREADS, sm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pseudo
