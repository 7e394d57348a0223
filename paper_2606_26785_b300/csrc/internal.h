// Launchers shared between the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"
#include "pseudo.h"

namespace pseudo {

// tri_kernels.cu
void launch_pack_panels(const double2 *T, int64_t ldT, int n, int n_pad, double2 *U64, double2 *L64,
                        float2 *U32, float2 *L32, cudaStream_t s);
int trsv_group_width(int fp32);
size_t trsv_scratch_bytes(int fp32, int64_t n_pad, int64_t ncols);
cudaError_t launch_trsv64(const double2 *Pn, int n, int n_pad, int lower, const int *cols, const double2 *zc,
                          int ncols, const int *ncols_dev, double2 *X, int64_t ldx, double2 *xs, cudaStream_t s);
// The same solve when only an upper bound of the column count is known on the
// host (the live count in *ncols_dev): the column-group widths the host
// version picks from the count are each launched over their range of counts.
cudaError_t launch_trsv64_bounded(const double2 *Pn, int n, int n_pad, int lower, const int *cols, const double2 *zc,
                                  int bound, const int *ncols_dev, double2 *X, int64_t ldx, double2 *xs,
                                  cudaStream_t s);
cudaError_t launch_trsv32(const float2 *Pn, int n, int n_pad, int lower, const int *cols, const double2 *zc,
                          int ncols, const int *ncols_dev, float2 *X, int64_t ldx, float2 *xs, cudaStream_t s);
cudaError_t launch_trmv64(const double2 *Pn, int n, int n_pad, int lower, const int *cols, const double2 *zc,
                          int ncols, const int *ncols_dev, const double2 *X, int64_t ldx, const double2 *B,
                          int64_t ldb, double2 *Y, int64_t ldy, int subtract, cudaStream_t s);
cudaError_t launch_trmv_ds(const float2 *Ph, const float2 *Pl, int n, int n_pad, int lower, const int *cols,
                           const double2 *zc, int ncols, const double2 *X, int64_t ldx, const double2 *B, int64_t ldb,
                           double2 *Y, int64_t ldy, int subtract, cudaStream_t s, float2 *Xh = nullptr,
                           float2 *Xl = nullptr);
void launch_pack_lo(const double2 *P64, const float2 *P32, float2 *Plo, int64_t cnt, cudaStream_t s);
cudaError_t launch_sumsq(const double2 *a, int64_t cnt, double *out, cudaStream_t s);
cudaError_t launch_extract_diag(const double2 *U, int n, int n_pad, double2 *d, cudaStream_t s);

}  // namespace pseudo

struct pseudo_ctx;
namespace pseudo {
// trsv_tc.cu: the tensor-core solve (row panels of 128; n_pad is a multiple of 128)
constexpr int TC_MB = 128;
size_t trsv32_scratch_bytes(int64_t n_pad, int64_t ncols);
int64_t tc_pack_floats(int n_pad);
int64_t tc_diag_elems(int n_pad);
void launch_pack_tc(const double2 *T, int64_t ldT, int n, int n_pad, float *AU, float *AL, float2 *DU, float2 *DL,
                    cudaStream_t s);
cudaError_t launch_trsv_tc(const pseudo_ctx *h, int lower, const int *cols, const double2 *zc, int ncols,
                           const int *ncols_dev, float2 *X, int64_t ldx, float2 *xs, cudaStream_t s);
// The FP32 multi-shift solve of the handle's choice (tensor cores or CUDA
// cores); xs is trsv_scratch_bytes(1, n_pad, ncols) of scratch.
cudaError_t solve32(const pseudo_ctx *h, int lower, const int *cols, const double2 *zc, int ncols,
                    const int *ncols_dev, float2 *X, int64_t ldx, float2 *xs, cudaStream_t s);
// unit roundoff of the FP32 solve in use (for the refinement plan)
double solve32_unit_roundoff(const pseudo_ctx *h);
// trsv_ds.cu: the multi-shift solve in double-single arithmetic (X is FP64 in
// and out; xs is trsv_ds_scratch_bytes(n_pad, ncols) of scratch)
size_t trsv_ds_scratch_bytes(int64_t n_pad, int64_t ncols);
cudaError_t launch_trsv_ds(const pseudo_ctx *h, int lower, const int *cols, const double2 *zc, int ncols,
                           const int *ncols_dev, double2 *X, int64_t ldx, void *xs, cudaStream_t s);
// trmv_oz.cu: double-single-accurate shifted products on the tensor cores
int64_t oz_a_elems(int n_pad);
size_t oz_scratch_bytes(int n_pad, int64_t ncols);
void launch_pack_oz(const double2 *T, int64_t ldT, int n, int n_pad, void *AU, void *AL, int *exU, int *exL,
                    cudaStream_t s);
cudaError_t launch_trmv_oz(const pseudo_ctx *h, int lower, const int *cols, const double2 *zc, int ncols,
                           const double2 *X, int64_t ldx, const double2 *B, int64_t ldb, double2 *Y, int64_t ldy,
                           int subtract, void *scratch, cudaStream_t s, const int *ncols_dev = nullptr);
}  // namespace pseudo

namespace pseudo {
// lanczos.cu
constexpr int LANCZOS_MMAX = 64;
void launch_start_vector(double2 *v, int n, uint64_t seed, cudaStream_t s);
template <typename real>
void launch_bcast_start(const double2 *v, int n, int S, cx_t<real> *Q0, cudaStream_t s);
template <typename real>
void launch_copy_cols(const cx_t<real> *src, cx_t<real> *dst, int n, int S, const int *active,
                      cudaStream_t s);
template <typename real>
void launch_lanczos_orth(cx_t<real> *Q, int64_t qs, cx_t<real> *W, int n, int S, int j, int mmax,
                         const int *active, double *alpha, double *beta, cudaStream_t s);
void launch_lanczos_tridiag(int S, int j, int mmax, const double *alpha, const double *beta, int *active,
                            double *theta, double *svec, int *nsteps, double tol_q, double tol_floor, int final_step,
                            cudaStream_t s);
void launch_compact_active(const int *active, int S, int *cols, int *cnt, cudaStream_t s);
template <typename real>
void launch_ritz_vector(const cx_t<real> *Q, int64_t qs, int n, int S, int mmax, const double *svec,
                        const int *nsteps, double2 *U, const int *mask, cudaStream_t s);
}  // namespace pseudo

namespace pseudo {
// colops.cu
void launch_colnorm2(const double2 *X, int n, int S, const int *mask, double *out, cudaStream_t s);
void launch_scale_to32(const double2 *R, int n, int S, const int *mask, const double *rn2, float2 *D, cudaStream_t s);
void launch_acc_from32(double2 *X, int n, int S, const int *mask, const double *rn2, const float2 *D, cudaStream_t s);
void launch_normalize(double2 *X, int n, int S, const int *mask, cudaStream_t s);
// s2 = ||Y||^2 over ny rows (0: n), r = ||NX - s2 U|| over n rows, per masked column
void launch_rq_residual(const double2 *U, const double2 *Y, const double2 *NX, int n, int S, const int *mask,
                        double *s2, double *r, cudaStream_t s, int ny = 0);
void launch_finalize(int S, int64_t w0, const double2 *z, const double *theta, const double *s2, const double *rr,
                     const int *active, const int *extra_flags, int sig_src, double norm2, const double *eps, int neps,
                     double *sigma_out, double *res_out, int32_t *flags_out, uint32_t *member_out, int base_flags,
                     int *nbad, cudaStream_t s);
void launch_fill_int(int *a, int n, int v, cudaStream_t s);
void launch_nonfinite(const double2 *a, int64_t cnt, int *bad, cudaStream_t s);
}  // namespace pseudo

namespace pseudo {
// tsk.cu: batched tall-skinny views. Item b's element (i, j) is p[b*bs + i*ld + j].
// With map != nullptr item b lives in slot map[b] (e.g. the recycle lane of a
// refined point).
// coff != nullptr adds a per-item element offset coff[b] (e.g. the column where
// a lane's new block starts).
struct TSView {
    double2 *p;
    int64_t ld, bs;
    const int *map;
    const int *coff;
    __host__ __device__ double2 *at(int b) const {
        return p + (int64_t)(map ? map[b] : b) * bs + (coff ? coff[b] : 0);
    }
};
inline TSView tsv(double2 *p, int64_t ld, int64_t bs, const int *map = nullptr, const int *coff = nullptr) {
    return TSView{p, ld, bs, map, coff};
}
cudaError_t launch_ts_gram(TSView A, int ka, TSView B, int kb, int n, int nitems, const int *items, double2 *G,
                           int64_t gstride, bool zero, cudaStream_t s);
cudaError_t launch_ts_mul(TSView A, int ka, const double2 *C, int64_t cstride, TSView O, int kb, int n, int nitems,
                          const int *items, double beta, double alpha, cudaStream_t s);
}  // namespace pseudo

namespace pseudo {
// recy_update.cu
void launch_upd_decide(const int *lanes, int nu, int *p, int r, int KM, int p_max, double omega, const double2 *C,
                       const double2 *gx, int *lout, int *kk, int *nskip, cudaStream_t s);
void launch_upd_shift(double2 *V, double2 *W1, double2 *W3, double2 *W4, int n, int64_t ld, double2 *H1, double2 *H2,
                      double2 *Lf, double2 *C, int KM, int r, const int *lanes, int nu, int *p, const int *lout,
                      cudaStream_t s);
void launch_upd_chol(const double2 *G, int r, int nu, const int *lout, double2 *R, double2 *Ri, cudaStream_t s);
void launch_upd_add(double2 *U, const double2 *U2, int cnt, int nu, cudaStream_t s);
void launch_upd_rotate(double2 *H1, double2 *H2, double2 *Lf, double2 *Qacc, const double2 *U, const double2 *Rnew,
                       const double2 *Hc1, const double2 *Hc2, const double2 *Hr2, int KM, int r, const int *lanes,
                       int nu, int *p, const int *kk, cudaStream_t s);
void launch_small_matmul(const double2 *A, const double2 *B, double2 *C, int m, int nitems, cudaStream_t s);
void launch_copy_block(TSView src, TSView dst, int n, int kc, int nitems, const int *items, cudaStream_t s);
}  // namespace pseudo

namespace pseudo {
// lanczos.cu: continuous batching (per-slot steps, refill on convergence)
template <typename real>
void launch_slot_copy(const cx_t<real> *Q, int64_t qs, cx_t<real> *W, int n, int S, const int *jv, const int *active,
                      cudaStream_t s);
template <typename real>
void launch_slot_orth(cx_t<real> *Q, int64_t qs, cx_t<real> *W, int n, int S, const int *jv, int mmax,
                      const int *active, double *alpha, double *beta, int passes, cudaStream_t s);
void launch_slot_tridiag(int S, int mmax, const double *alpha, const double *beta, int *active, int *jv, double *theta,
                         double *svec, int *convd, double tol_q, double tol_floor, int fp32, cudaStream_t s);
template <typename real>
void launch_slot_harvest(cx_t<real> *Q, int64_t qs, int n, int S, int mmax, const double *svec, int *jv, int *active,
                         const double *theta, const int *convd, int *pt, double2 *zslot, const double2 *zall, int npts,
                         int *counters, double2 *Ufin, int F, int *fin_pt, double2 *fin_z, double *fin_theta,
                         int *fin_conv, const double2 *v0, int4 *work, cudaStream_t s, const double2 *vw = nullptr,
                         int64_t ldw = 0, const int *posw = nullptr, int offw = 0);
// fallback points (fb_list != NULL) get column t of U0 (n x ldu) copied to
// column k of warm (n x ldw) when warm != NULL, k = their place in fb_list
void launch_fin_scatter(int P, const int *fin_pt, const double2 *fin_z, const double *fin_theta, const int *fin_conv,
                        const double *s2, const double *rr, int use_rq, double norm2, const double *eps, int neps,
                        double *sigma_out, double *res_out, int32_t *flags_out, uint32_t *member_out, int *nbad,
                        double u_solve, double fb_ku, int *fb_list, int *fb_cnt, cudaStream_t s,
                        const double2 *U0 = nullptr, int64_t ldu = 0, double2 *warm = nullptr, int64_t ldw = 0,
                        int n = 0, const double2 *v0 = nullptr, const int *P_dev = nullptr);
void launch_mask_prefix(int *mask, int F, const int *P, cudaStream_t s);
// rect.cu: rectangular input (m = 2n)
int64_t rect_packed_size(int n);
int rect_max_order();  // largest n of a rectangular pencil (shared-memory right-hand sides)
cudaError_t launch_rect_qr(const pseudo_ctx *h, const int *cols, int ncols, const int *ncols_dev,
                           const double2 *zslot, double2 *Rz, double2 *Rs, double2 *Bs, cudaStream_t s);
cudaError_t launch_rect_solve(const pseudo_ctx *h, const double2 *Rs, int lower, const int *cols, int ncols,
                              const int *ncols_dev, double2 *X, int64_t ldx, cudaStream_t s);
void launch_add_cols(double2 *A, const double2 *B, int64_t cnt, cudaStream_t s);
cudaError_t rect_normal_product(pseudo_ctx *h, const double2 *zc, int ncols, const int *ncols_dev, const double2 *X,
                                int64_t ldx, double2 *Y, int64_t ldy, double2 *NX, double2 *Tb, cudaStream_t s);
void launch_lanc_ctrl(const int *cnt, const int *counters, int S, const int *err, long long guard, long long *ctl,
                      long long *stat, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hf,
                      cudaGraphConditionalHandle hs, int graph, cudaStream_t s);
void launch_fb_gather(const int *list, int cnt, const double2 *zall, double2 *zc, cudaStream_t s);
void launch_fb_scatter(const int *list, int cnt, const double *sc, const double *rc, const int32_t *fc,
                       const uint32_t *mc, double *sigma, double *res, int32_t *flags, uint32_t *member,
                       cudaStream_t s);
}  // namespace pseudo

namespace pseudo {
template <typename real>
void launch_slot_orth_grid(cx_t<real> *Q, int64_t qs, cx_t<real> *W, int n, int S, const int *jv, int mmax,
                           const int *active, double *alpha, double *beta, int passes, double2 *Hp, double *nrm2,
                           double *alpha_acc, cudaStream_t s);
}  // namespace pseudo
