// Handle layout, workspace carving and grid-driver entry points (host side).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

#include "pseudo.h"
#include "internal.h"

namespace pseudo {
// A named range on a profiler's NVTX timeline for the scope it lives in (the
// phases of the grid drivers, named as in the paper's time breakdown); it does
// nothing when no profiler is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
struct GraphCache;  // instantiated device-loop graphs of a handle (invlanc.cu)
constexpr int RECY_KMAX = 64;  // largest recycled rank k = p_max * r supported
int set_err(int code, const char *fmt, ...);
int cuda_err(cudaError_t e, const char *where);
void clear_err();
// true when p is not a multiple of a (a power of two); NULL is aligned
bool misaligned(const void *p, uintptr_t a);
// the tuned table of autotune_table.h: FP32 solver kernel and Lanczos slots for order n
int tuned_fp32_solver(int n);
int tuned_slots(int n);

// Bump allocator over the caller's workspace (256-byte aligned pieces).  With
// a null base it only measures.
struct Carver {
    char *base = nullptr;
    size_t cap = 0, used = 0;
    bool overflow = false;
    Carver() {}
    Carver(char *b, size_t c) : base(b), cap(c) {}
    void *take(size_t bytes);
    template <typename T> T *get(size_t count) { return (T *)take(count * sizeof(T)); }
};

struct GridIO {
    const double2 *z;
    int64_t npts;
    const double *eps_host;
    int neps;
    double *sigma, *res;
    int32_t *flags;
    uint32_t *member;
    bool on_host;
};
}  // namespace pseudo

#include <vector>

struct pseudo_ctx {
    int dev = 0;
    // per-kernel-class profiling (pseudo_opts.profile)
    struct KRec {
        int cls, ea, eb;
        double flops, bytes;
    };
    bool prof = false;
    std::vector<cudaEvent_t> evs;
    int evn = 0;
    std::vector<KRec> recs;
    pseudo_kstat kst[PSEUDO_K_COUNT] = {};
    int n = 0, n_pad = 0;
    double2 *U64 = nullptr, *L64 = nullptr;  // packed panels of T and T^H, FP64
    float2 *U32 = nullptr, *L32 = nullptr;   // the same in FP32 (the high parts)
    float2 *U32lo = nullptr, *L32lo = nullptr;  // fl32(T - fl32(T)): low parts for double-single products
    double2 *diag = nullptr;                 // T_ii (the eigenvalues of C)
    // tensor-core solve: A'' chunks (TF32 hi/lo, shared-memory image) and
    // FP32 diagonal blocks of T and T^H; device error word of bounded waits
    float *tcA_U = nullptr, *tcA_L = nullptr;
    float2 *tcD_U = nullptr, *tcD_L = nullptr;
    int *dev_err = nullptr;                  // [0] a bounded wait gave up, [1] scratch flag of argument checks
    uint64_t wait_ns = 1000000000ull;        // limit of every bounded wait in the tensor-core kernels
    // tensor-core double-single products: 7 bf16 slices of T and T^H per
    // (64-row tile, 16-column chunk) image, and the per-row scale exponents
    void *ozA_U = nullptr, *ozA_L = nullptr;
    int *ozE_U = nullptr, *ozE_L = nullptr;
    int fp32_solver = 0;                     // 0 tensor cores (form by order), 1 CUDA cores,
                                             // PSEUDO_SOLVER_TC16 / TC32 tensor cores in that form
    // rectangular input (m = 2n, SM2.2): M = [T; B] dense column-major (2n x n,
    // leading dimension 2n) and the FP64 panels of B and B^H
    bool rect = false;
    double2 *M64 = nullptr, *BU64 = nullptr, *BL64 = nullptr;
    pseudo::GraphCache *graph_cache = nullptr;
    double norm_fro = 0.0, norm2 = 0.0;      // ||T||_F and a 2-norm estimate
    pseudo_stats_t stats;
};

namespace pseudo {
inline int kp_begin(pseudo_ctx *h, cudaStream_t s) {
    if (!h->prof) return -1;
    if (h->evn >= (int)h->evs.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        h->evs.push_back(e);
    }
    cudaEventRecord(h->evs[h->evn], s);
    return h->evn++;
}
inline void kp_end(pseudo_ctx *h, int ea, int cls, double flops, double bytes, cudaStream_t s) {
    if (ea < 0) return;
    const int eb = kp_begin(h, s);
    h->recs.push_back({cls, ea, eb, flops, bytes});
}
// After the stream has been synchronised: fold the event pairs into kst.
inline void kp_resolve(pseudo_ctx *h) {
    for (const auto &r : h->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->evs[r.ea], h->evs[r.eb]);
        h->kst[r.cls].launches += 1;
        h->kst[r.cls].ms += ms;
        h->kst[r.cls].flops += r.flops;
        h->kst[r.cls].bytes += r.bytes;
    }
    h->recs.clear();
    h->evn = 0;
}
// algorithmic work of one multi-shift solve / product launch on ncols columns
inline double tri_flops(int n, int ncols) { return 4.0 * (double)n * n * ncols; }
inline double tri_bytes(int n, int ncols, double tri_esz, double vec_esz, int nvec) {
    return 0.5 * (double)n * n * tri_esz + (double)nvec * n * ncols * vec_esz;
}

void invlanc_carve(pseudo_ctx *h, const pseudo_opts *o, int64_t npts, Carver &c, void *plan);
void graph_cache_free(pseudo_ctx *h);
int invlanc_run(pseudo_ctx *h, const pseudo_opts *o, const GridIO &io, Carver &c, cudaStream_t s);
void recycle_carve(pseudo_ctx *h, const pseudo_opts *o, int64_t npts, Carver &c, void *plan);
int recycle_run(pseudo_ctx *h, const pseudo_opts *o, const GridIO &io, Carver &c, cudaStream_t s);
void recycle_state_layout(pseudo_ctx *h, const pseudo_opts *o, int64_t npts, int64_t *out);
void launch_convert_64_to_32(const double2 *a, float2 *b, int64_t cnt, cudaStream_t s);
void launch_convert_32_to_64(const float2 *a, double2 *b, int64_t cnt, cudaStream_t s);
}  // namespace pseudo

namespace pseudo {
// (T - zI)^{op} products for the refinement residuals and the recycled
// subspace: IEEE FP64 in FP64 mode, double-single on the FP32 units in mixed
// mode.  With ncols_dev the launch covers ncols columns (an upper bound) and
// the kernels read the live count from device memory.
// xh / xl: scratch with X's layout (leading dimension ldx) for the FP32 split
// of X used by the double-single kernel.
inline cudaError_t trmv_hp(pseudo_ctx *h, bool ds, int lower, const int *cols, const double2 *zc, int ncols,
                           const double2 *X, int64_t ldx, const double2 *B, int64_t ldb, double2 *Y, int64_t ldy,
                           int subtract, cudaStream_t s, float2 *xh = nullptr, float2 *xl = nullptr,
                           void *oz = nullptr, const int *ncols_dev = nullptr) {
    if (ds && oz && h->ozA_U)
        return launch_trmv_oz(h, lower, cols, zc, ncols, X, ldx, B, ldb, Y, ldy, subtract, oz, s, ncols_dev);
    if (ds) {
        if (ncols_dev) return cudaErrorInvalidValue;  // the CUDA-core double-single product takes host counts only
        return launch_trmv_ds(lower ? h->L32 : h->U32, lower ? h->L32lo : h->U32lo, h->n, h->n_pad, lower, cols, zc,
                              ncols, X, ldx, B, ldb, Y, ldy, subtract, s, xh, xl);
    }
    return launch_trmv64(lower ? h->L64 : h->U64, h->n, h->n_pad, lower, cols, zc, ncols, ncols_dev, X, ldx, B, ldb, Y,
                         ldy, subtract, s);
}
}  // namespace pseudo

namespace pseudo {
// refine.cu: iterative refinement of shifted solves (mixed precision)
struct IRBufs {
    double2 *R64;     // residuals, n x S
    float2 *D32;      // FP32 right-hand sides / corrections, n x S
    double *rn2;      // per-column squared residual norms
    int *mask, *need, *perm;
    float2 *xs;       // FP32 solve scratch for S columns
    float2 *xh, *xl;  // double-single split of X, n x S
    void *oz;         // tensor-core product scratch (oz_scratch_bytes for S columns) or NULL
};
struct IRPlan {
    std::vector<int> cnt;  // cnt[it]: columns still refining at step it
};
// need[c] for c < sig.size(), zero for the other columns up to S_total and for
// the columns marked in *skip (their solution stays zero)
void ir_plan(pseudo_ctx *h, const std::vector<double> &sig, const std::vector<double2> &z, int max_ir,
             const IRBufs &b, IRPlan &plan, cudaStream_t s, int S_total = 0, const std::vector<char> *skip = nullptr);
cudaError_t ir_solve_cols(pseudo_ctx *h, const IRBufs &b, int lower, const double2 *zc, int S, const double2 *B,
                          double2 *X, const IRPlan &plan, cudaStream_t s);
// The same plan made on the device for the *nfin finished columns of a
// capacity-F buffer (Lanczos values theta, shifts z, convergence flags conv):
// need/perm in b, cnt[0 .. max_ir] (device); stat[0] and stat[1] (device)
// accumulate the solves and products it implies.
void ir_plan_dev(pseudo_ctx *h, const int *nfin, int F, const double *theta, const double2 *z, const int *conv,
                 int max_ir, double fb_ku, const IRBufs &b, int *cnt, long long *stat, cudaStream_t s);
// Refinement under a device plan: max_ir launches of each kind whose column
// counts come from cnt, so that the launch sequence is fixed (capturable).
cudaError_t ir_solve_cols_dev(pseudo_ctx *h, const IRBufs &b, int lower, const double2 *zc, int S, const double2 *B,
                              double2 *X, int max_ir, const int *cnt, cudaStream_t s);
}  // namespace pseudo

