// CTA-cooperative small dense FP64 routines on shared-memory matrices
// (row-major, leading dimension = order).  Every thread of the CTA must call
// them (they synchronise internally).  FP64 throughput on this GPU is low per
// instruction, so each routine spreads its work over all threads instead of
// running a scalar loop in one thread.
#pragma once
#include "common.cuh"

namespace pseudo {

// Round-robin (tournament) pairing of m (even) indices: pair q of round rd.
__device__ __forceinline__ void rr_pair(int m, int rd, int q, int &a, int &b) {
    auto at = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + rd) % (m - 1)) + 1; };
    a = at(q);
    b = at(m - 1 - q);
    if (a > b) { int t = a; a = b; b = t; }
}

// Hermitian eigen-decomposition by cyclic two-sided Jacobi: H (k x k, only
// read as Hermitian) is overwritten; on return diag(H) holds the eigenvalues
// (unsorted) and G (k x k) the eigenvectors as columns.  rot: >= 192 doubles.
// Rotation for the pair (p, q) with h = H_pq = |h| e^{i phi}:
//   J = [[c, s], [-s e^{-i phi}, c e^{-i phi}]],  tau = (H_qq - H_pp)/(2|h|),
//   t = sign(tau)/(|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2), s = t c;
// H <- J^H H J zeroes H_pq, G <- G J.
static __device__ void blk_heev_jacobi(double2 *H, double2 *G, int k, double *rot, int max_sweeps = 40) {
    const double tol = 4e-16 * k;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < k * k; e += nt) G[e] = make_double2((e / k) == (e % k) ? 1.0 : 0.0, 0.0);
    __shared__ double s_off;
    __syncthreads();
    if (k <= 1) return;
    const int m = (k + 1) & ~1;
    double *rc = rot, *rs = rot + 32, *rer = rot + 64, *rei = rot + 96, *rt = rot + 128;
    int *rpq = (int *)(rot + 160);
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        // convergence: max |H_pq| / sqrt(|H_pp H_qq|)
        if (tid == 0) s_off = 0.0;
        __syncthreads();
        double loc = 0.0;
        for (int e = tid; e < k * k; e += nt) {
            const int p = e / k, q = e % k;
            if (p < q) {
                const double hpq = sqrt(cabs2(H[e]));
                const double den = sqrt(fabs(H[p * k + p].x) * fabs(H[q * k + q].x));
                const double r = den > 0.0 ? hpq / den : (hpq > 0.0 ? 1.0 : 0.0);
                loc = fmax(loc, r);
            }
        }
        for (int o = 16; o > 0; o >>= 1) loc = fmax(loc, __shfl_xor_sync(0xffffffffu, loc, o));
        if ((tid & 31) == 0) atomicMax((unsigned long long *)&s_off, __double_as_longlong(loc));
        __syncthreads();
        if (s_off <= tol) break;
        for (int rd = 0; rd < m - 1; ++rd) {
            if (tid < m / 2) {
                int p, q;
                rr_pair(m, rd, tid, p, q);
                double c = 1.0, s = 0.0, er = 1.0, ei = 0.0, t = 0.0;
                if (q < k) {
                    const double2 h = H[p * k + q];
                    const double g = sqrt(cabs2(h));
                    const double hpp = H[p * k + p].x, hqq = H[q * k + q].x;
                    if (g > 1e-300 && g > tol * sqrt(fabs(hpp * hqq))) {
                        const double tau = (hqq - hpp) / (2.0 * g);
                        t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                        er = h.x / g; ei = -h.y / g;  // e^{-i phi}
                    }
                }
                rc[tid] = c; rs[tid] = s; rer[tid] = er; rei[tid] = ei; rt[tid] = t;
                rpq[2 * tid] = p; rpq[2 * tid + 1] = q;
            }
            __syncthreads();
            // rows: H <- J^H H ; row_p' = c row_p - s e^{i phi} row_q ; row_q' = s row_p + c e^{i phi} row_q
            for (int e = tid; e < (m / 2) * k; e += nt) {
                const int pi = e / k, j = e % k;
                const int p = rpq[2 * pi], q = rpq[2 * pi + 1];
                if (q >= k || rs[pi] == 0.0) continue;
                const double c = rc[pi], s = rs[pi];
                const double2 eip = make_double2(rer[pi], -rei[pi]);  // e^{+i phi}
                const double2 hp = H[p * k + j], hq = H[q * k + j];
                const double2 eq = cmul(eip, hq);
                H[p * k + j] = make_double2(c * hp.x - s * eq.x, c * hp.y - s * eq.y);
                H[q * k + j] = make_double2(s * hp.x + c * eq.x, s * hp.y + c * eq.y);
            }
            __syncthreads();
            // columns: H <- H J, G <- G J ; col_p' = c col_p - s e^{-i phi} col_q ; col_q' = s col_p + c e^{-i phi} col_q
            for (int e = tid; e < (m / 2) * k * 2; e += nt) {
                const int which = e / ((m / 2) * k);
                const int ee = e % ((m / 2) * k);
                const int pi = ee / k, i = ee % k;
                const int p = rpq[2 * pi], q = rpq[2 * pi + 1];
                if (q >= k || rs[pi] == 0.0) continue;
                double2 *X = which ? G : H;
                const double c = rc[pi], s = rs[pi];
                const double2 emi = make_double2(rer[pi], rei[pi]);
                const double2 xp = X[i * k + p], xq = X[i * k + q];
                const double2 eq = cmul(emi, xq);
                X[i * k + p] = make_double2(c * xp.x - s * eq.x, c * xp.y - s * eq.y);
                X[i * k + q] = make_double2(s * xp.x + c * eq.x, s * xp.y + c * eq.y);
            }
            __syncthreads();
            if (tid < m / 2) {
                const int p = rpq[2 * tid], q = rpq[2 * tid + 1];
                if (q < k && rs[tid] != 0.0) {
                    H[p * k + q] = make_double2(0.0, 0.0);
                    H[q * k + p] = make_double2(0.0, 0.0);
                    H[p * k + p].y = 0.0;
                    H[q * k + q].y = 0.0;
                }
            }
            __syncthreads();
        }
    }
}

// Ascending order of the real diagonal of H (k x k): perm[0..k) and vals.
static __device__ void blk_sort_diag(const double2 *H, int k, int *perm, double *vals) {
    const int tid = threadIdx.x;
    for (int i = tid; i < k; i += blockDim.x) {
        const double v = H[i * k + i].x;
        int rank = 0;
        for (int j = 0; j < k; ++j) {
            const double w = H[j * k + j].x;
            rank += (w < v) || (w == v && j < i);
        }
        perm[rank] = i;
        vals[rank] = v;
    }
    __syncthreads();
}

// One-sided Jacobi SVD of the m x m matrix A (row-major, columns rotated in
// place): on return the column norms of A are the singular values and Vr
// (m x m) holds the right singular vectors as columns (A_in Vr = A_out).
// red: >= 2*m*m doubles + 160 doubles of scratch.
static __device__ void blk_svd_jacobi(double2 *A, double2 *Vr, int m, double *red, int max_sweeps = 40) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < m * m; e += nt) Vr[e] = make_double2((e / m) == (e % m) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    if (m <= 1) return;
    const int mm = (m + 1) & ~1, half = mm / 2;
    double *pa = red, *pb = red + 32, *pgr = red + 64, *pgi = red + 96;
    int *pp = (int *)(red + 128);
    __shared__ double s_off;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (tid == 0) s_off = 0.0;
        __syncthreads();
        for (int rd = 0; rd < mm - 1; ++rd) {
            if (tid < half) {
                int p, q;
                rr_pair(mm, rd, tid, p, q);
                pp[2 * tid] = p; pp[2 * tid + 1] = q;
                double a = 0, b = 0, gr = 0, gi = 0;
                if (q < m) {
                    for (int i = 0; i < m; ++i) {
                        const double2 x = A[i * m + p], y = A[i * m + q];
                        a += cabs2(x); b += cabs2(y);
                        gr += x.x * y.x + x.y * y.y;
                        gi += x.x * y.y - x.y * y.x;
                    }
                }
                pa[tid] = a; pb[tid] = b; pgr[tid] = gr; pgi[tid] = gi;
            }
            __syncthreads();
            for (int e = tid; e < half * m * 2; e += nt) {
                const int which = e / (half * m);
                const int ee = e % (half * m);
                const int pi = ee / m, i = ee % m;
                const int p = pp[2 * pi], q = pp[2 * pi + 1];
                if (q >= m) continue;
                const double a = pa[pi], b = pb[pi];
                const double g = sqrt(pgr[pi] * pgr[pi] + pgi[pi] * pgi[pi]);
                if (a == 0.0 || b == 0.0 || g == 0.0 || g <= 1e-16 * sqrt(a) * sqrt(b)) continue;
                const double zeta = (b - a) / (2.0 * g);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                const double2 emi = make_double2(pgr[pi] / g, -pgi[pi] / g);
                double2 *X = which ? Vr : A;
                const double2 xp = X[i * m + p], xq = X[i * m + q];
                const double2 eq = cmul(emi, xq);
                X[i * m + p] = make_double2(c * xp.x - s * eq.x, c * xp.y - s * eq.y);
                X[i * m + q] = make_double2(s * xp.x + c * eq.x, s * xp.y + c * eq.y);
            }
            if (tid < half) {
                const int q = pp[2 * tid + 1];
                if (q < m) {
                    const double a = pa[tid], b = pb[tid];
                    const double g = sqrt(pgr[tid] * pgr[tid] + pgi[tid] * pgi[tid]);
                    const double r = (a > 0 && b > 0) ? g / sqrt(a) / sqrt(b) : 0.0;
                    if (r > 0.0) atomicMax((unsigned long long *)&s_off, __double_as_longlong(r));
                }
            }
            __syncthreads();
        }
        if (s_off <= 1e-15) break;
    }
}

// Column norms of A (m x m) into sig[m].
static __device__ void blk_colnorms(const double2 *A, int m, double *sig) {
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += cabs2(A[i * m + j]);
        sig[j] = sqrt(s);
    }
    __syncthreads();
}

// Cholesky of the Hermitian positive definite m x m matrix A (upper factor R,
// A = R^H R, written in place, strictly lower part zeroed).  Returns false
// (to every thread) if a pivot is not positive.
static __device__ bool blk_cholesky(double2 *A, int m) {
    __shared__ int s_ok;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) s_ok = 1;
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        if (tid == 0) {
            const double d = A[j * m + j].x;
            if (!(d > 0.0)) s_ok = 0;
            A[j * m + j] = make_double2(d > 0.0 ? sqrt(d) : 1.0, 0.0);
        }
        __syncthreads();
        const double inv = 1.0 / A[j * m + j].x;
        for (int c = j + 1 + tid; c < m; c += nt) { A[j * m + c].x *= inv; A[j * m + c].y *= inv; }
        __syncthreads();
        // trailing update: A[a][b] -= conj(R[j][a]) R[j][b] for j < a <= b
        for (int e = tid; e < m * m; e += nt) {
            const int a = e / m, b = e % m;
            if (a > j && b >= a) cfms(A[a * m + b], cconj(A[j * m + a]), A[j * m + b]);
        }
        __syncthreads();
    }
    for (int e = tid; e < m * m; e += nt)
        if (e / m > e % m) A[e] = make_double2(0.0, 0.0);
    __syncthreads();
    return s_ok != 0;
}

// Inverse of the upper-triangular m x m R into Ri (upper).  Column-parallel
// back substitution: column c of Ri solves R x = e_c.
static __device__ void blk_triu_inverse(const double2 *R, double2 *Ri, int m) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) Ri[e] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        for (int i = c; i >= 0; --i) {
            double2 s = make_double2(i == c ? 1.0 : 0.0, 0.0);
            for (int l = i + 1; l <= c; ++l) cfms(s, R[i * m + l], Ri[l * m + c]);
            Ri[i * m + c] = cmul(s, crecip(R[i * m + i]));
        }
    }
    __syncthreads();
}

}  // namespace pseudo
