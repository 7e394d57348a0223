// Multi-shift triangular solve on the 5th-generation tensor cores (tcgen05):
// (T - z_c I) x_c = b_c or (T - z_c I)^H x_c = b_c for many columns c at once,
// the FP32 form of the R(z)^{-1} / R(z)^{-*} applications (Alg. 3, the
// inverse-Lanczos comparator and the refinement solves).
//
// The shift only touches the diagonal, so every off-diagonal block product
// T_IK x_K is shared by all shifts and is a plain complex GEMM.  A CTA owns
// NC right-hand sides and walks row panels of 128 rows (bottom-up for T,
// top-down for T^H).  For a panel, D = sum_K T_IK X_K over the solved rows is
// accumulated in TMEM by tcgen05.mma (kind::tf32, M = 128, N = 2 NC), then
// the 128 x 128 shifted diagonal block is solved on the CUDA cores in FP32
// (one row per thread, one column of the block per step).
//
// Complex as real: with A'' = [Re T_IK  Im T_IK] (128 x 2KC) and
// B'' = [[Re X, Im X], [-Im X, Re X]] (2KC x 2NC), A'' B'' = [Re, Im] of T_IK X_K.
// FP32 accuracy from TF32 units ("3xTF32"): every operand is split into
// hi = tf32(v) and lo = tf32(v - hi), and A''B'' ~ hi hi + hi lo + lo hi.
// A'' is split and packed once (at handle creation) in exactly the byte image
// the MMA reads from shared memory, so a chunk is one bulk copy; B'' is built
// from the solved columns by the CTA's threads.
#include <cmath>

#include "common.cuh"
#include "driver.h"
#include "internal.h"
#include "tc.cuh"

namespace pseudo {

namespace {
constexpr int MB = 128;               // panel rows (MMA M)
constexpr int KC = 16;                // complex K per chunk
constexpr int KR = 2 * KC;            // real K per chunk
constexpr int A_SPLIT = MB * KR;      // floats of one split of an A chunk
constexpr int A_CHUNK = 2 * A_SPLIT;  // hi + lo

__host__ __device__ __forceinline__ int64_t chunk_base(int64_t p) { return 4 * p * (p - 1); }
}  // namespace

int64_t tc_pack_floats(int n_pad) {
    const int64_t P = n_pad / MB;
    return chunk_base(P) * A_CHUNK;
}
int64_t tc_diag_elems(int n_pad) { return (int64_t)(n_pad / MB) * MB * MB; }

// A'' chunks of every panel in processing order; see the file comment.
__global__ void pack_tc_a_kernel(const double2 *__restrict__ T, int64_t ldT, int n, int n_pad, int lower,
                                 float *__restrict__ out, int64_t total) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int P = n_pad / MB;
    const int64_t qq = e / A_CHUNK;
    const int w = (int)(e % A_CHUNK);
    const int split = w / A_SPLIT, ww = w % A_SPLIT;
    const int cmi = ww >> 5, r7 = (ww >> 2) & 7, k3 = ww & 3;
    const int kb = cmi / (MB / 8), rb = cmi % (MB / 8);
    const int m = rb * 8 + r7, kk = kb * 4 + k3;
    int64_t p = (int64_t)((1.0 + sqrt(1.0 + (double)qq)) * 0.5);
    while (p > 1 && chunk_base(p) > qq) --p;
    while (chunk_base(p + 1) <= qq) ++p;
    const int t = (int)(qq - chunk_base(p));
    const int J = lower ? (int)p : P - 1 - (int)p;
    const int k0 = lower ? KC * t : n_pad - KC * (t + 1);
    const int row = J * MB + m, kc = k0 + (kk % KC), part = kk / KC;
    double comp = 0.0;
    if (row < n && kc < n) {
        if (!lower) {
            if (row <= kc) { const double2 v = T[(int64_t)kc * ldT + row]; comp = part ? v.y : v.x; }
        } else {
            if (kc <= row) { const double2 v = T[(int64_t)row * ldT + kc]; comp = part ? -v.y : v.x; }
        }
    }
    const float f = (float)comp;
    const float hi = tc::to_tf32(f);
    out[e] = split ? tc::to_tf32(f - hi) : hi;
}

// Diagonal blocks, step-major: D[J][j][i] is the coefficient of x_j in row i
// of block J: T(i, j) for the upper solve, conj(T(j, i)) for the lower one.
__global__ void pack_tc_d_kernel(const double2 *__restrict__ T, int64_t ldT, int n, int n_pad,
                                 float2 *__restrict__ DU, float2 *__restrict__ DL) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)(n_pad / MB) * MB * MB) return;
    const int J = (int)(e / (MB * MB)), w = (int)(e % (MB * MB));
    const int j = w / MB, i = w % MB;
    const int ri = J * MB + i, rj = J * MB + j;
    float2 u = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
    if (ri < n && rj < n) {
        if (i <= j) { const double2 v = T[(int64_t)rj * ldT + ri]; u = make_float2((float)v.x, (float)v.y); }
        if (j <= i) { const double2 v = T[(int64_t)ri * ldT + rj]; l = make_float2((float)v.x, (float)-v.y); }
    }
    DU[e] = u;
    DL[e] = l;
}

void launch_pack_tc(const double2 *T, int64_t ldT, int n, int n_pad, float *AU, float *AL, float2 *DU, float2 *DL,
                    cudaStream_t s) {
    const int64_t tot = tc_pack_floats(n_pad);
    if (tot > 0) {
        const unsigned bl = (unsigned)((tot + 255) / 256);
        note_launch(); pack_tc_a_kernel<<<bl, 256, 0, s>>>(T, ldT, n, n_pad, 0, AU, tot);
        note_launch(); pack_tc_a_kernel<<<bl, 256, 0, s>>>(T, ldT, n, n_pad, 1, AL, tot);
    }
    const int64_t nd = tc_diag_elems(n_pad);
    note_launch(); pack_tc_d_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(T, ldT, n, n_pad, DU, DL);
}

// Warp roles of the solve (256 threads):
//   warp 0      : producer     - per chunk, one bulk copy of the packed A''
//                                chunk and one of the B'' image of the solved
//                                rows it multiplies, into a ring of NS stages
//                                (chunks of the panel just solved wait for it);
//   warp 1      : MMA issuer   - for every chunk, 12 tcgen05.mma into the
//                                panel's TMEM accumulator (two accumulators,
//                                so the next panel starts while the current
//                                one is being solved);
//   warps 4-7   : diagonal     - read the accumulator (one row per thread), form
//                                b - D, solve the shifted 128 x 128 diagonal
//                                block, write the rows out and the B'' images
//                                (TF32 hi/lo, MMA byte order) of the new rows.
// Hand-offs are mbarriers; every wait is bounded and gives up on a shared
// abort flag.  Warps 2-3 only take part in set-up and tear-down.
namespace {
// Two configurations of (columns per CTA, ring stages):
//   narrow: 16 columns, 2 stages of 40 KB, two CTAs per SM;
//   wide:   32 columns, 4 stages of 48 KB, one CTA per SM; the reciprocal
//           diagonal shares the accumulator's turnaround buffer to make room.
// At large orders a CTA's sweep is set by its stream of chunks (about 0.6 us
// per chunk whether 37 or 148 CTAs run, and whether the ring has 3 or 4
// stages), and a wide chunk carries twice the columns for 1.2x the bytes, so a
// wide CTA finishes its 32 columns sooner than a narrow CTA its 16: measured
// at n = 8000, 1.16x (1,184 columns) to 1.31x (9,472 columns) faster; at
// n = 4000, 1.12x.  At small orders the 128-step diagonal-block solves set
// the pace instead, and a wide CTA has twice the columns per diagonal warp:
// at n = 256 .. 2048 the narrow form is 1.2-1.6x faster, so handles below
// TC_WIDE_MIN_NPAD keep it.
#ifndef TC_WIDE_STAGES
#define TC_WIDE_STAGES 4   // ring stages of the wide form (3 measured the same; 4 is the most that fits)
#endif
constexpr int NC_NARROW = 16, NS_NARROW = 2;
constexpr int NC_WIDE = 32, NS_WIDE = TC_WIDE_STAGES;
#ifndef TC_WIDE_MIN_NPAD
#define TC_WIDE_MIN_NPAD 4096   // padded order from which a handle uses the wide configuration
#endif
#ifndef TC_NACC
#define TC_NACC 1   // partial accumulators per panel (more did not pay off when measured)
#endif
#ifndef TC_PD
#define TC_PD 4   // prefetch distance of the diagonal-block coefficients (steps)
#endif
#ifndef TC_A_EVICT_LAST
#define TC_A_EVICT_LAST 1   // A chunks copied with an L2 evict-last policy (every CTA streams them)
#endif
constexpr int TC_THREADS = 256;
constexpr int BAR_DIAG = 1;  // named barrier of the diagonal warps (0 is __syncthreads)

__device__ __forceinline__ void named_bar(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
// bounded wait (limit_ns) that also gives up as soon as another role has aborted
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort,
                                              uint64_t limit_ns) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = tc::global_ns();
    for (;;) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (tc::global_ns() - t0 > limit_ns) { *abort = 1; return false; }
    }
}
}  // namespace

template <int NC, int NS>
struct TcSmem {
    // the wide form keeps 1 / (t_ii - z_c) in the turnaround buffer once the
    // accumulator has been read out of it; the narrow form has its own array
    static constexpr bool dinv_shared = NC >= 32;
    static constexpr int NR = 2 * NC;            // real N of the MMA
    static constexpr int B_SPLIT = NR * KR;      // floats
    static constexpr int B_IMG = 2 * B_SPLIT;    // hi + lo
    static constexpr size_t stage = (size_t)(A_CHUNK + B_IMG) * sizeof(float);
    // ring of stages, then the turned-around accumulator and 1 / (t_ii - z_c)
    static constexpr size_t diag =
        (size_t)MB * (2 * NC + 1) * sizeof(float) + (dinv_shared ? 0 : (size_t)MB * NC * sizeof(float2));
    static constexpr size_t bytes = NS * stage + diag + 128;  // + alignment slack
    // two panels in flight, TC_NACC partial accumulators each (power of two >= 32 columns)
    static constexpr uint32_t acc_cols = 2 * TC_NACC * NR;
    static constexpr uint32_t tmem_cols = acc_cols <= 32 ? 32 : acc_cols <= 64 ? 64 : acc_cols <= 128 ? 128
                                          : acc_cols <= 256 ? 256 : 512;
};

// Scratch of the solves for ncols columns: the compact copy of each column
// group's solution (the CUDA-core kernel, groups of 16) followed by the B''
// images of every 16-row chunk of each group (the tensor-core kernel, groups
// of 16 or 32 columns).  Both cost 40 bytes per column and row, so the layout
// of the wider groups (ncols rounded up to 32) covers every kernel.
size_t trsv32_scratch_bytes(int64_t n_pad, int64_t ncols) {
    static_assert(NC_WIDE % NC_NARROW == 0 && NC_NARROW % 16 == 0, "groups nest");
    const int64_t groups = (ncols + NC_WIDE - 1) / NC_WIDE;
    return (size_t)groups * n_pad * NC_WIDE * sizeof(float2) +
           (size_t)groups * (n_pad / KC) * TcSmem<NC_WIDE, NS_WIDE>::B_IMG * sizeof(float);
}

template <int NC, int NS>
__global__ void __launch_bounds__(TC_THREADS, NS <= 2 && NC <= 16 ? 2 : 1)
trsv_tc_kernel(const float *__restrict__ Apack, const float2 *__restrict__ Dblk, int n, int n_pad, int lower,
               const int *__restrict__ cols, const double2 *__restrict__ zc, int ncols_host,
               const int *__restrict__ ncols_dev, float2 *X, int64_t ldx, float2 *xs_all, int *err,
               uint64_t wait_ns) {
    using L = TcSmem<NC, NS>;
    static_assert(L::bytes + 1024 <= 227 * 1024, "ring and turnaround buffers exceed the shared memory of a CTA");
    constexpr int NR = L::NR;
    constexpr int LBO_A = (MB / 8) * 128, LBO_B = (NR / 8) * 128;
    static_assert(NR % 32 == 0, "the diagonal warps read the accumulator in 32-column pieces");
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[NS], freeb[NS];
    __shared__ __align__(8) uint64_t acc_full[2], acc_free[2], solved;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ int s_flag_diag;
    __shared__ int s_col[NC];
    __shared__ float2 s_z[NC];
    __shared__ int s_last_ld, s_last_mma;

    const int ncols = ncols_dev ? *ncols_dev : ncols_host;
    const int g = blockIdx.x;
    if (g * NC >= ncols) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float *sbuf = reinterpret_cast<float *>(smem_raw + ((128 - (tc::smem_u32(smem_raw) & 127)) & 127));
    constexpr int STAGE_F = A_CHUNK + L::B_IMG;  // floats per stage: A'' hi, A'' lo, B'' hi, B'' lo
    // B'' images of this group: one per 16-row chunk, after every group's compact copy
    float *bimg = reinterpret_cast<float *>(xs_all + (int64_t)gridDim.x * n_pad * NC) +
                  (int64_t)g * (n_pad / KC) * L::B_IMG;

    if (tid < NC) {
        const int pos = g * NC + tid;
        int c = -1;
        double2 z = make_double2(0.0, 0.0);
        if (pos < ncols) { c = cols ? cols[pos] : pos; z = zc[c]; }
        if (lower) z.y = -z.y;  // (T - zI)^H = T^H - conj(z) I
        s_col[tid] = c;
        s_z[tid] = make_float2((float)z.x, (float)z.y);
    }
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) { tc::mbar_init(&full[i], 1); tc::mbar_init(&freeb[i], 1); }
        for (int i = 0; i < 2; ++i) { tc::mbar_init(&acc_full[i], 1); tc::mbar_init(&acc_free[i], 1); }
        tc::mbar_init(&solved, 1);
        tc::mbar_fence_init();
        s_abort = 0;
        s_last_ld = -1;
        s_last_mma = -1;
    }
    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, L::tmem_cols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;
    const int P = n_pad / MB;

    if (warp == 0) {
        // -------------------------------------------------------- producer
        if (lane == 0) {
            int q = 0, known = 0;  // panels known to be solved
            const uint64_t keep = tc::l2_policy_evict_last();  // every CTA streams the same A chunks
            for (int p = 0; p < P && !s_abort; ++p) {
                const float *Ap = Apack + chunk_base(p) * A_CHUNK;
                bool ok = true;
                for (int t = 0; t < 8 * p; ++t, ++q) {
                    const int st = q % NS;
                    const int k0 = lower ? KC * t : n_pad - KC * (t + 1);
                    const int pk = lower ? k0 / MB : P - 1 - k0 / MB;  // processing index of those rows' panel
                    if (pk >= known) {
                        if (!wait_or_abort(&solved, pk & 1, &s_abort, wait_ns)) { ok = false; break; }
                        known = pk + 1;
                    }
                    if (q >= NS && !wait_or_abort(&freeb[st], ((q / NS) - 1) & 1, &s_abort, wait_ns)) { ok = false; break; }
                    float *dst = sbuf + st * STAGE_F;
                    tc::mbar_expect_tx(&full[st], (uint32_t)L::stage);
                    if (TC_A_EVICT_LAST)
                        tc::bulk_g2s_hint(dst, Ap + (int64_t)t * A_CHUNK, A_CHUNK * sizeof(float), &full[st], keep);
                    else
                        tc::bulk_g2s(dst, Ap + (int64_t)t * A_CHUNK, A_CHUNK * sizeof(float), &full[st]);
                    tc::bulk_g2s(dst + A_CHUNK, bimg + (int64_t)(k0 / KC) * L::B_IMG, L::B_IMG * sizeof(float),
                                 &full[st]);
                    s_last_ld = q;
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_tf32(MB, NR);
            const uint32_t s0 = tc::smem_u32(sbuf);
            int q = 0;
            for (int p = 0; p < P && !s_abort; ++p) {
                const int buf = p & 1;
                if (p >= 2 && !wait_or_abort(&acc_free[buf], ((p >> 1) - 1) & 1, &s_abort, wait_ns)) break;
                tc::tc_fence_after();
                const uint32_t dacc = tmem + buf * (TC_NACC * NR);
                const int nch = 8 * p;
                bool ok = true;
                for (int t = 0; t < nch; ++t, ++q) {
                    const int st = q % NS;
                    if (!wait_or_abort(&full[st], (q / NS) & 1, &s_abort, wait_ns)) { ok = false; break; }
                    tc::tc_fence_after();
                    const uint32_t ah = s0 + st * (STAGE_F * 4), al = ah + A_SPLIT * 4;
                    const uint32_t bh = ah + A_CHUNK * 4, bl = bh + L::B_SPLIT * 4;
#pragma unroll
                    for (int ks = 0; ks < KR / 8; ++ks) {
                        const uint64_t dah = tc::smem_desc(ah + ks * 2 * LBO_A, LBO_A, 128);
                        const uint64_t dal = tc::smem_desc(al + ks * 2 * LBO_A, LBO_A, 128);
                        const uint64_t dbh = tc::smem_desc(bh + ks * 2 * LBO_B, LBO_B, 128);
                        const uint64_t dbl = tc::smem_desc(bl + ks * 2 * LBO_B, LBO_B, 128);
                        // consecutive MMAs go to different partial accumulators so that
                        // they do not wait on each other; the diagonal warps add them up
                        constexpr int NA = TC_NACC;
                        const int g3 = (3 * ks) % NA;
                        tc::mma_tf32(dacc + ((g3 + 0) % NA) * NR, dah, dbh, idesc, (t == 0 && 3 * ks + 0 < NA) ? 0u : 1u);
                        tc::mma_tf32(dacc + ((g3 + 1) % NA) * NR, dah, dbl, idesc, (t == 0 && 3 * ks + 1 < NA) ? 0u : 1u);
                        tc::mma_tf32(dacc + ((g3 + 2) % NA) * NR, dal, dbh, idesc, (t == 0 && 3 * ks + 2 < NA) ? 0u : 1u);
                    }
                    tc::mma_commit(&freeb[st]);
                    s_last_mma = q;
                }
                if (!ok) break;
                if (nch > 0) tc::mma_commit(&acc_full[buf]);
                else mbar_arrive(&acc_full[buf]);
            }
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------ diagonal solve
        // The accumulator arrives one row per thread (TMEM lane = row); it is
        // turned around through shared memory so that each warp owns NC/4
        // columns of all 128 rows (rows lane + 32k, k = 0..3) and solves them
        // on its own: one shuffle broadcast per step and no block barrier in
        // the 128 steps.
        constexpr int CPW = NC / 4;
        const int i = tid - 128, dw = warp - 4;
        const int cw0 = dw * CPW;
        float *Dsm = sbuf + NS * STAGE_F;                 // [MB][2 NC + 1]
        float2 *s_dinv = reinterpret_cast<float2 *>(L::dinv_shared ? Dsm : Dsm + MB * (2 * NC + 1));  // [MB][NC]
        for (int p = 0; p < P; ++p) {
            const int J = lower ? p : P - 1 - p;
            const int buf = p & 1;
            if (i == 0) s_flag_diag = wait_or_abort(&acc_full[buf], (p >> 1) & 1, &s_abort, wait_ns) ? 1 : 0;
            named_bar(BAR_DIAG, 128);
            if (!s_flag_diag) break;
            tc::tc_fence_after();
            const float2 *DJ = Dblk + (int64_t)J * MB * MB;
            {   // row i: accumulator into shared memory, and 1 / (t_ii - z_c)
#pragma unroll
                for (int piece = 0; piece < NR / 32; ++piece) {
                    float d[32];
#pragma unroll
                    for (int u = 0; u < 32; ++u) d[u] = 0.f;
                    if (p > 0) {
                        // panels with fewer than TC_NACC MMAs leave the later
                        // accumulators unwritten: only the ones in use are read
                        const int used = min(TC_NACC, 8 * p * 3 * (KR / 8));
                        for (int a = 0; a < used; ++a) {
                            float e[32];
                            tc::tmem_ld32(tmem + buf * (TC_NACC * NR) + a * NR + piece * 32 +
                                          ((uint32_t)(dw * 32) << 16), e);
#pragma unroll
                            for (int u = 0; u < 32; ++u) d[u] += e[u];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 32; ++u) Dsm[i * (2 * NC + 1) + piece * 32 + u] = d[u];
                }
                if constexpr (!L::dinv_shared) {
                    const float2 tii = DJ[i * MB + i];
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        s_dinv[i * NC + c] = crecip(make_float2(tii.x - s_z[c].x, tii.y - s_z[c].y));
                }
            }
            tc::tc_fence_before();
            named_bar(BAR_DIAG, 128);
            if (i == 0) mbar_arrive(&acc_free[buf]);
            // this warp's columns cw0 .. cw0 + CPW - 1, rows lane + 32 k
            float2 r[4][CPW];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int rl = lane + 32 * k, row = J * MB + rl;
#pragma unroll
                for (int c = 0; c < CPW; ++c) {
                    const int col = cw0 + c;
                    float2 b = make_float2(0.f, 0.f);
                    if (row < n && s_col[col] >= 0) b = X[(int64_t)row * ldx + s_col[col]];
                    r[k][c] = make_float2(b.x - Dsm[rl * (2 * NC + 1) + col], b.y - Dsm[rl * (2 * NC + 1) + NC + col]);
                }
            }
            if constexpr (L::dinv_shared) {
                // every warp has read its part of the accumulator: the buffer
                // now takes the reciprocal diagonal (row i, all NC columns)
                named_bar(BAR_DIAG, 128);
                const float2 tii = DJ[i * MB + i];
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    s_dinv[i * NC + c] = crecip(make_float2(tii.x - s_z[c].x, tii.y - s_z[c].y));
                named_bar(BAR_DIAG, 128);
            }
            // coefficient of x_j in this thread's rows, loaded PD steps ahead
            // (the stored blocks are zero where a row does not depend on x_j)
            constexpr int PD = TC_PD;
            float2 pf[PD][4];
#pragma unroll
            for (int u = 0; u < PD; ++u) {
                const int j = lower ? u : MB - 1 - u;
#pragma unroll
                for (int k = 0; k < 4; ++k) pf[u][k] = DJ[j * MB + lane + 32 * k];
            }
#pragma unroll
            for (int kq = 0; kq < 4; ++kq) {              // the 32-row slot of the step's row
                const int kj = lower ? kq : 3 - kq;
                for (int blk = 0; blk < 32 / PD; ++blk) {
#pragma unroll
                    for (int u = 0; u < PD; ++u) {
                        const int lj = lower ? blk * PD + u : 31 - (blk * PD + u);
                        const int j = 32 * kj + lj;
                        float2 t[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) t[k] = pf[u][k];
                        const int jn = lower ? j + PD : j - PD;
                        if (jn >= 0 && jn < MB) {
#pragma unroll
                            for (int k = 0; k < 4; ++k) pf[u][k] = DJ[jn * MB + lane + 32 * k];
                        }
                        // x_j for this warp's columns: computed from lane lj's row, broadcast
#pragma unroll
                        for (int c = 0; c < CPW; ++c) {
                            const float2 xo = cmul(r[kj][c], s_dinv[j * NC + cw0 + c]);
                            const float2 xb = shfl_c(xo, lj);
                            if (lane == lj) r[kj][c] = xb;
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                if (k != kj || lane != lj) cfms(r[k][c], t[k], xb);
                        }
                    }
                }
            }
            // the rows out, and their B'' = [[Re x, Im x], [-Im x, Re x]] image
            // (hi and lo TF32 splits) for the chunks of later panels
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int rl = lane + 32 * k, row = J * MB + rl;
                const int kl = rl % KC;
                float *bh = bimg + (int64_t)(row / KC) * L::B_IMG, *bl = bh + L::B_SPLIT;
#pragma unroll
                for (int c = 0; c < CPW; ++c) {
                    const int col = cw0 + c;
                    const float2 v = row < n ? r[k][c] : make_float2(0.f, 0.f);
                    if (row < n && s_col[col] >= 0) X[(int64_t)row * ldx + s_col[col]] = v;
                    const float vv[4] = {v.x, -v.y, v.y, v.x};
                    const int jj[4] = {col, col, NC + col, NC + col};
                    const int kk[4] = {kl, KC + kl, kl, KC + kl};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float h = tc::to_tf32(vv[e]);
                        const int o = tc::cm_index(jj[e], kk[e], NR);
                        bh[o] = h;
                        bl[o] = tc::to_tf32(vv[e] - h);
                    }
                }
            }
            tc::fence_async_global();
            __threadfence_block();
            named_bar(BAR_DIAG, 128);
            if (i == 0) mbar_arrive(&solved);
        }
    }
    // ---- teardown (also after an abort: let copies and MMAs in flight finish)
    __syncthreads();
    if (tid == 0 && s_abort) {
        // copies still in flight are among the last NS issued (a stage is
        // reloaded only after its MMAs are done); none of those stages has been
        // re-armed since, so each wait below ends when its copy lands
        const int ql = s_last_ld, qm = s_last_mma;
        for (int q = ql - NS + 1 < 0 ? 0 : ql - NS + 1; q <= ql; ++q)
            tc::mbar_wait(&full[q % NS], (q / NS) & 1, 100000000ull);
        if (qm >= 0) tc::mbar_wait(&freeb[qm % NS], (qm / NS) & 1, 100000000ull);
        atomicExch(err, 1);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, L::tmem_cols);
}

template <int NC, int NS>
static cudaError_t launch_tc(const pseudo_ctx *h, int lower, const int *cols, const double2 *zc, int ncols,
                             const int *ncols_dev, float2 *X, int64_t ldx, float2 *xs, cudaStream_t s) {
    using L = TcSmem<NC, NS>;
    static std::atomic<uint64_t> attr{0};
    smem_attr_once(trsv_tc_kernel<NC, NS>, (int)L::bytes, attr);
    const int grid = (ncols + NC - 1) / NC;
    if (grid == 0) return cudaSuccess;
    note_launch();
    trsv_tc_kernel<NC, NS><<<grid, TC_THREADS, L::bytes, s>>>(lower ? h->tcA_L : h->tcA_U, lower ? h->tcD_L : h->tcD_U,
                                                             h->n, h->n_pad, lower, cols, zc, ncols, ncols_dev, X, ldx,
                                                             xs, h->dev_err, h->wait_ns);
    return cudaGetLastError();
}

// the FP32 solver codes that run the tensor-core solve (pseudo_opts.fp32_solver)
static bool tc_solver(int code) { return code == 0 || code == PSEUDO_SOLVER_TC16 || code == PSEUDO_SOLVER_TC32; }

cudaError_t launch_trsv_tc(const pseudo_ctx *h, int lower, const int *cols, const double2 *zc, int ncols,
                           const int *ncols_dev, float2 *X, int64_t ldx, float2 *xs, cudaStream_t s) {
    const bool wide = h->fp32_solver == PSEUDO_SOLVER_TC32 ||
                      (h->fp32_solver != PSEUDO_SOLVER_TC16 && h->n_pad >= TC_WIDE_MIN_NPAD);
    if (wide)
        return launch_tc<NC_WIDE, NS_WIDE>(h, lower, cols, zc, ncols, ncols_dev, X, ldx, xs, s);
    return launch_tc<NC_NARROW, NS_NARROW>(h, lower, cols, zc, ncols, ncols_dev, X, ldx, xs, s);
}

cudaError_t solve32(const pseudo_ctx *h, int lower, const int *cols, const double2 *zc, int ncols,
                    const int *ncols_dev, float2 *X, int64_t ldx, float2 *xs, cudaStream_t s) {
    // the scratch (trsv32_scratch_bytes) covers every kernel's column groups
    if (tc_solver(h->fp32_solver) && h->tcA_U)
        return launch_trsv_tc(h, lower, cols, zc, ncols, ncols_dev, X, ldx, xs, s);
    return launch_trsv32(lower ? h->L32 : h->U32, h->n, h->n_pad, lower, cols, zc, ncols, ncols_dev, X, ldx, xs, s);
}

// 3xTF32 products carry about 2^-22 relative error against FP32's 2^-24
double solve32_unit_roundoff(const pseudo_ctx *h) {
    return (tc_solver(h->fp32_solver) && h->tcA_U) ? 2.4e-7 : 5.96e-8;
}

}  // namespace pseudo
