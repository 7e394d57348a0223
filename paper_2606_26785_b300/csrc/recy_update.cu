// Adaptive update of the recycling subspace (Alg. 2, updateRecy), batched
// over recycle lanes.  Lane arrays V, W1 = T V, W3 = T^H T V, W4 = T^H V are
// n x (lanes * KM) row-major (lane l owns columns [l KM, l KM + KM)), columns
// beyond a lane's k = p r are kept at zero; H1 = W1^H W1, H2 = W1^H V and the
// block lower-triangular factor L of [X^1 .. X^p] = V L (eq. (QLfact)) are
// KM x KM per lane.  The n-space products run through the batched
// tall-skinny kernels and the triangular product kernel; this file holds the
// k-space steps:
//   upd_decide : rho_j = ||(I - V_j V_j^H) x_1|| from c = V^H x_1 (rho_j^2 =
//                ||x_1||^2 - sum over the kept tail |c_t|^2, monotone in j),
//                l = the last j with rho_j <= omega rho_0 (eq. (omegaCond)),
//                raised so that at most p_max blocks remain.
//   upd_shift  : drop the first l blocks of V, W1, W3, W4 (n-space) and of
//                H1, H2, L (k-space).
//   upd_chol   : R and R^{-1} of the CholeskyQR of the orthogonalised block.
//   upd_rotate : append the new block column [U_{.,new}; U_{new,new}] to L
//                (eq. (blkGS)) and annihilate U_{j,new}, j = 1..p-l, by the
//                block-unitary 2r x 2r transforms Q_j (Householder QR of
//                [U_{new,new}; U_{j,new}]), applied to L, H1, H2 and
//                accumulated into Q = prod Q_j, which the driver then applies
//                to V, W1, W3, W4 in n-space.
#include "common.cuh"
#include "internal.h"
#include "recycle.h"
#include "smalldense.cuh"

namespace pseudo {

constexpr int UP_THREADS = 256;

// Per updating lane u (lane id lanes[u]):
//   C  : KM x r  = V^H X (rows >= k are zero),  gx : r x r = X^H X
//   out: l[u] (blocks dropped, -1 = skip the append), kk[u] = (p - l) r
__global__ void upd_decide_kernel(const int *__restrict__ lanes, int *__restrict__ p, int r, int KM, int p_max,
                                  double omega, const double2 *__restrict__ C, const double2 *__restrict__ gx,
                                  int *__restrict__ lout, int *__restrict__ kkout, int *__restrict__ nskip) {
    const int u = blockIdx.x;
    if (threadIdx.x != 0) return;
    const int lane = lanes[u];
    const int pp = p[lane], k = pp * r;
    const double2 *Cu = C + (int64_t)u * KM * r;
    const double x2 = gx[(int64_t)u * r * r].x;  // ||x_1||^2
    double tail = 0.0;                            // sum_{t >= jr} |c_t|^2, built from the back
    double tails[65];
    tails[pp] = 0.0;
    for (int j = pp - 1; j >= 0; --j) {
        for (int t = j * r; t < (j + 1) * r; ++t) tail += cabs2(Cu[t * r]);
        tails[j] = tail;
    }
    const double rho0 = sqrt(fmax(x2 - tails[0], 0.0));
    int l;
    if (pp > 0 && rho0 <= 1e-12 * sqrt(x2)) {
        l = -1;  // x_1 already in span V: nothing to append
        atomicAdd(nskip, 1);
    } else {
        l = pp;
        for (int j = 1; j <= pp; ++j) {
            const double rhoj = sqrt(fmax(x2 - tails[j], 0.0));
            if (rhoj > omega * rho0) { l = j - 1; break; }
        }
        if (pp - l + 1 > p_max) l = pp + 1 - p_max;
    }
    (void)k;
    lout[u] = l;
    kkout[u] = l < 0 ? -1 : (pp - l) * r;
}

// Drop the first l blocks (lb = l r columns) of a lane's V, W1, W3, W4: one
// thread per row moves the row left in ascending column order (safe in place)
// and zeroes the freed tail.
__global__ void upd_shift_n_kernel(double2 *__restrict__ V, double2 *__restrict__ W1, double2 *__restrict__ W3,
                                   double2 *__restrict__ W4, int n, int64_t ld, int KM, int r,
                                   const int *__restrict__ lanes, const int *__restrict__ p,
                                   const int *__restrict__ lout) {
    const int u = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = lout[u];
    if (i >= n || l <= 0) return;
    const int lane = lanes[u];
    const int k = p[lane] * r, lb = l * r;
    double2 *M[4] = {V, W1, W3, W4};
    for (int q = 0; q < 4; ++q) {
        double2 *row = M[q] + (int64_t)i * ld + (int64_t)lane * KM;
        for (int c = 0; c + lb < k; ++c) row[c] = row[c + lb];
        for (int c = k - lb; c < k; ++c) row[c] = make_double2(0.0, 0.0);
    }
}

// Drop the first l blocks of H1, H2, L (k-space) and set p <- p - l; also
// keep rows lb.. of C (the BCGS coefficients) as rows 0.. .
__global__ void upd_shift_k_kernel(double2 *__restrict__ H1, double2 *__restrict__ H2, double2 *__restrict__ Lf,
                                   double2 *__restrict__ C, int KM, int r, const int *__restrict__ lanes,
                                   int *__restrict__ p, const int *__restrict__ lout) {
    const int u = blockIdx.x;
    const int l = lout[u];
    const int lane = lanes[u];
    const int k = p[lane] * r;
    if (l > 0) {
        const int lb = l * r, kn = k - lb;
        double2 *M[3] = {H1 + (int64_t)lane * KM * KM, H2 + (int64_t)lane * KM * KM, Lf + (int64_t)lane * KM * KM};
        for (int q = 0; q < 3; ++q) {
            // move rows/cols [lb, k) to [0, kn): ascending order, one pass per row
            for (int a = 0; a < kn; ++a) {
                // source row a + lb and destination row a differ, so each thread
                // can move its elements without waiting on the others
                for (int b = threadIdx.x; b < kn; b += blockDim.x) M[q][a * KM + b] = M[q][(a + lb) * KM + b + lb];
                __syncthreads();
            }
            for (int e = threadIdx.x; e < KM * KM; e += blockDim.x) {
                const int a = e / KM, b = e % KM;
                if (a >= kn || b >= kn) M[q][e] = make_double2(0.0, 0.0);
            }
            __syncthreads();
        }
        double2 *Cu = C + (int64_t)u * KM * r;
        for (int a = 0; a < kn; ++a) {
            for (int c = threadIdx.x; c < r; c += blockDim.x) Cu[a * r + c] = Cu[(a + lb) * r + c];
            __syncthreads();
        }
        for (int e = threadIdx.x; e < KM * r; e += blockDim.x)
            if (e / r >= kn) Cu[e] = make_double2(0.0, 0.0);
        __syncthreads();
        if (threadIdx.x == 0) p[lane] -= l;
    }
}

// R (upper) and R^{-1} of the column-scaled Cholesky of the r x r Gram.
__global__ void __launch_bounds__(UP_THREADS)
upd_chol_kernel(const double2 *__restrict__ G, int r, const int *__restrict__ lout, double2 *__restrict__ R,
                double2 *__restrict__ Ri) {
    __shared__ double2 A[64], B[64];
    __shared__ double d[8];
    const int u = blockIdx.x;
    if (lout && lout[u] < 0) return;
    const int tid = threadIdx.x;
    for (int e = tid; e < r * r; e += blockDim.x) A[e] = G[(int64_t)u * r * r + e];
    __syncthreads();
    if (tid < r) d[tid] = sqrt(fmax(A[tid * r + tid].x, 0.0));
    __syncthreads();
    for (int e = tid; e < r * r; e += blockDim.x) {
        const int a = e / r, b = e % r;
        const double s = d[a] * d[b];
        A[e] = s > 0.0 ? cscale(A[e], 1.0 / s) : make_double2(a == b ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    if (!blk_cholesky(A, r)) {
        // shifted retry
        for (int e = tid; e < r * r; e += blockDim.x) {
            const int a = e / r, b = e % r;
            const double s = d[a] * d[b];
            A[e] = s > 0.0 ? cscale(G[(int64_t)u * r * r + e], 1.0 / s) : make_double2(a == b ? 1.0 : 0.0, 0.0);
            if (a == b) A[e].x += 1e-13 * r;
        }
        __syncthreads();
        blk_cholesky(A, r);
    }
    for (int e = tid; e < r * r; e += blockDim.x) A[e] = cscale(A[e], d[e % r] > 0.0 ? d[e % r] : 1.0);
    __syncthreads();
    blk_triu_inverse(A, B, r);
    for (int e = tid; e < r * r; e += blockDim.x) {
        R[(int64_t)u * r * r + e] = A[e];
        Ri[(int64_t)u * r * r + e] = B[e];
    }
}

// U += U2 (second BCGS pass coefficients), both KM x r per lane
__global__ void upd_add_kernel(double2 *__restrict__ U, const double2 *__restrict__ U2, int cnt) {
    const int u = blockIdx.x;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        double2 a = U[(int64_t)u * cnt + e];
        const double2 b = U2[(int64_t)u * cnt + e];
        a.x += b.x; a.y += b.y;
        U[(int64_t)u * cnt + e] = a;
    }
}

// Householder QR of the 2r x r block Y (smem, ld r) producing the explicit
// 2r x 2r unitary Q (ld 2r) with Y = Q [R; 0].
static __device__ void house_qr_2r(double2 *Y, double2 *Q, int r, double2 *vbuf) {
    const int m = 2 * r, tid = threadIdx.x;
    __shared__ double s_beta;
    for (int e = tid; e < m * m; e += blockDim.x) Q[e] = make_double2((e / m) == (e % m) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    for (int c = 0; c < r; ++c) {
        if (tid == 0) {
            double nrm2 = 0.0;
            for (int i = c; i < m; ++i) nrm2 += cabs2(Y[i * r + c]);
            const double nrm = sqrt(nrm2);
            const double2 x0 = Y[c * r + c];
            const double ax0 = sqrt(cabs2(x0));
            double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
            // alpha = -ph * nrm; v = x - alpha e_1
            for (int i = 0; i < m; ++i) vbuf[i] = make_double2(0.0, 0.0);
            for (int i = c; i < m; ++i) vbuf[i] = Y[i * r + c];
            vbuf[c].x += ph.x * nrm;
            vbuf[c].y += ph.y * nrm;
            double vv = 0.0;
            for (int i = c; i < m; ++i) vv += cabs2(vbuf[i]);
            s_beta = vv > 0.0 ? 2.0 / vv : 0.0;
        }
        __syncthreads();
        const double beta = s_beta;
        // Y <- (I - beta v v^H) Y for columns >= c ; Q <- Q (I - beta v v^H)
        for (int j = c + tid; j < r; j += blockDim.x) {
            double2 s = make_double2(0.0, 0.0);
            for (int i = c; i < m; ++i) cfma(s, cconj(vbuf[i]), Y[i * r + j]);
            s = cscale(s, beta);
            for (int i = c; i < m; ++i) cfms(Y[i * r + j], vbuf[i], s);
        }
        for (int i = tid; i < m; i += blockDim.x) {
            double2 s = make_double2(0.0, 0.0);
            for (int t = c; t < m; ++t) cfma(s, Q[i * m + t], vbuf[t]);
            s = cscale(s, beta);
            for (int t = c; t < m; ++t) cfms(Q[i * m + t], s, cconj(vbuf[t]));
        }
        __syncthreads();
    }
}

// Append the new block column of L and restore its block lower-triangular
// form; H1, H2 get their new blocks (already computed into Hc1 = W1^H W1_new
// (KM x r), Hc2 = W1^H V_new (KM x r), Hr2 = W1_new^H V (r x KM)) and every
// rotation; Qacc (KM x KM per lane) receives the product of the rotations.
__global__ void __launch_bounds__(UP_THREADS)
upd_rotate_kernel(double2 *__restrict__ H1, double2 *__restrict__ H2, double2 *__restrict__ Lf,
                  double2 *__restrict__ Qacc, const double2 *__restrict__ U, const double2 *__restrict__ Rnew,
                  const double2 *__restrict__ Hc1, const double2 *__restrict__ Hc2, const double2 *__restrict__ Hr2,
                  int KM, int r, const int *__restrict__ lanes, int *__restrict__ p, const int *__restrict__ kkv) {
    __shared__ double2 Y[16 * 8], Q[16 * 16], vbuf[16];
    __shared__ double2 tmp[2 * 8 * 64];
    const int u = blockIdx.x;
    const int kk = kkv[u];
    const int tid = threadIdx.x;
    const int lane = lanes[u];
    double2 *h1 = H1 + (int64_t)lane * KM * KM, *h2 = H2 + (int64_t)lane * KM * KM, *L = Lf + (int64_t)lane * KM * KM;
    double2 *Qa = Qacc + (int64_t)u * KM * KM;
    for (int e = tid; e < KM * KM; e += blockDim.x) Qa[e] = make_double2((e / KM) == (e % KM) ? 1.0 : 0.0, 0.0);
    if (kk < 0) return;
    const int kn = kk + r;  // new k
    const double2 *Uu = U + (int64_t)u * KM * r, *Ru = Rnew + (int64_t)u * r * r;
    const double2 *c1 = Hc1 + (int64_t)u * KM * r, *c2 = Hc2 + (int64_t)u * KM * r, *r2 = Hr2 + (int64_t)u * r * KM;
    // new block column of L, and new blocks of H1 (Hermitian) and H2
    for (int e = tid; e < kn * r; e += blockDim.x) {
        const int a = e / r, c = e % r;
        L[a * KM + kk + c] = a < kk ? Uu[a * r + c] : Ru[(a - kk) * r + c];
        const double2 v1 = c1[a * r + c];
        h1[a * KM + kk + c] = v1;
        h1[(kk + c) * KM + a] = cconj(v1);
        h2[a * KM + kk + c] = c2[a * r + c];
    }
    for (int e = tid; e < r * kk; e += blockDim.x) {
        const int c = e / kk, b = e % kk;
        h2[(kk + c) * KM + b] = r2[c * KM + b];
    }
    for (int e = tid; e < r * kk; e += blockDim.x) {  // new block row of L is zero left of the diagonal block
        const int c = e / kk, b = e % kk;
        L[(kk + c) * KM + b] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    // rotations j = 0 .. p-l-1 (old blocks); the new block is rows/cols [kk, kn)
    const int nb = kk / r;
    for (int j = 0; j < nb; ++j) {
        const int jr = j * r;
        for (int e = tid; e < 2 * r * r; e += blockDim.x) {
            const int i = e / r, c = e % r;
            Y[i * r + c] = i < r ? L[(kk + i) * KM + kk + c] : L[(jr + i - r) * KM + kk + c];
        }
        __syncthreads();
        house_qr_2r(Y, Q, r, vbuf);
        // rows: [L_new; L_j] <- Q^H [L_new; L_j]  (all kn columns), same for H1, H2 rows
        double2 *Ms[3] = {L, h1, h2};
        for (int q = 0; q < 3; ++q) {
            for (int e = tid; e < 2 * r * kn; e += blockDim.x) {
                const int i = e / kn, b = e % kn;
                double2 s = make_double2(0.0, 0.0);
                for (int t = 0; t < 2 * r; ++t) {
                    const int row = t < r ? kk + t : jr + t - r;
                    cfma(s, cconj(Q[t * 2 * r + i]), Ms[q][row * KM + b]);
                }
                tmp[e] = s;
            }
            __syncthreads();
            for (int e = tid; e < 2 * r * kn; e += blockDim.x) {
                const int i = e / kn, b = e % kn;
                const int row = i < r ? kk + i : jr + i - r;
                Ms[q][row * KM + b] = tmp[e];
            }
            __syncthreads();
        }
        // columns: H1, H2 <- (.) Q ; Qacc <- Qacc Q
        double2 *Mc[3] = {h1, h2, Qa};
        for (int q = 0; q < 3; ++q) {
            const int rows = q == 2 ? KM : kn;
            for (int e = tid; e < rows * 2 * r; e += blockDim.x) {
                const int a = e / (2 * r), i = e % (2 * r);
                double2 s = make_double2(0.0, 0.0);
                for (int t = 0; t < 2 * r; ++t) {
                    const int col = t < r ? kk + t : jr + t - r;
                    cfma(s, Mc[q][a * KM + col], Q[t * 2 * r + i]);
                }
                tmp[e] = s;
            }
            __syncthreads();
            for (int e = tid; e < rows * 2 * r; e += blockDim.x) {
                const int a = e / (2 * r), i = e % (2 * r);
                const int col = i < r ? kk + i : jr + i - r;
                Mc[q][a * KM + col] = tmp[e];
            }
            __syncthreads();
        }
        // exact zeros where the transform annihilated U_{j,new}
        for (int e = tid; e < r * r; e += blockDim.x) {
            const int i = e / r, c = e % r;
            L[(jr + i) * KM + kk + c] = make_double2(0.0, 0.0);
        }
        __syncthreads();
    }
    if (tid == 0) p[lane] = kn / r;
}

// C_b = A_b B_b for m x m blocks (item stride m*m)
__global__ void small_matmul_kernel(const double2 *__restrict__ A, const double2 *__restrict__ B, double2 *__restrict__ C,
                                    int m) {
    const int b = blockIdx.x;
    const double2 *Ab = A + (int64_t)b * m * m, *Bb = B + (int64_t)b * m * m;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        double2 s = make_double2(0.0, 0.0);
        for (int t = 0; t < m; ++t) cfma(s, Ab[i * m + t], Bb[t * m + j]);
        C[(int64_t)b * m * m + e] = s;
    }
}

// dst block <- src block (n x kc) per item
__global__ void copy_block_kernel(TSView src, TSView dst, int n, int kc, const int *__restrict__ items) {
    const int b = items ? items[blockIdx.y] : blockIdx.y;
    const double2 *sp = src.at(b);
    double2 *dp = dst.at(b);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * kc;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / kc, c = e % kc;
        dp[i * dst.ld + c] = sp[i * src.ld + c];
    }
}

// ------------------------------------------------------------ launchers
void launch_small_matmul(const double2 *A, const double2 *B, double2 *C, int m, int nitems, cudaStream_t s) {
    if (nitems > 0) { note_launch(); small_matmul_kernel<<<nitems, 64, 0, s>>>(A, B, C, m); }
}
void launch_copy_block(TSView src, TSView dst, int n, int kc, int nitems, const int *items, cudaStream_t s) {
    if (nitems <= 0 || kc <= 0) return;
    dim3 g(64, nitems);
    note_launch(); copy_block_kernel<<<g, 256, 0, s>>>(src, dst, n, kc, items);
}
void launch_upd_decide(const int *lanes, int nu, int *p, int r, int KM, int p_max, double omega, const double2 *C,
                       const double2 *gx, int *lout, int *kk, int *nskip, cudaStream_t s) {
    if (nu > 0) { note_launch(); upd_decide_kernel<<<nu, 32, 0, s>>>(lanes, p, r, KM, p_max, omega, C, gx, lout, kk, nskip); }
}
void launch_upd_shift(double2 *V, double2 *W1, double2 *W3, double2 *W4, int n, int64_t ld, double2 *H1, double2 *H2,
                      double2 *Lf, double2 *C, int KM, int r, const int *lanes, int nu, int *p, const int *lout,
                      cudaStream_t s) {
    if (nu <= 0) return;
    dim3 g((n + 127) / 128, nu);
    note_launch(); upd_shift_n_kernel<<<g, 128, 0, s>>>(V, W1, W3, W4, n, ld, KM, r, lanes, p, lout);
    note_launch(); upd_shift_k_kernel<<<nu, 256, 0, s>>>(H1, H2, Lf, C, KM, r, lanes, p, lout);
}
void launch_upd_chol(const double2 *G, int r, int nu, const int *lout, double2 *R, double2 *Ri, cudaStream_t s) {
    if (nu > 0) { note_launch(); upd_chol_kernel<<<nu, UP_THREADS, 0, s>>>(G, r, lout, R, Ri); }
}
void launch_upd_add(double2 *U, const double2 *U2, int cnt, int nu, cudaStream_t s) {
    if (nu > 0) { note_launch(); upd_add_kernel<<<nu, 128, 0, s>>>(U, U2, cnt); }
}
void launch_upd_rotate(double2 *H1, double2 *H2, double2 *Lf, double2 *Qacc, const double2 *U, const double2 *Rnew,
                       const double2 *Hc1, const double2 *Hc2, const double2 *Hr2, int KM, int r, const int *lanes,
                       int nu, int *p, const int *kk, cudaStream_t s) {
    if (nu > 0)
        note_launch(); upd_rotate_kernel<<<nu, UP_THREADS, 0, s>>>(H1, H2, Lf, Qacc, U, Rnew, Hc1, Hc2, Hr2, KM, r, lanes, p, kk);
}

}  // namespace pseudo
