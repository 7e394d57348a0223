// Handle layout, workspace carving and grid-driver entry points (host side).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "pseudo.h"

namespace pseudo {
constexpr int RECY_KMAX = 64;  // largest recycled rank k = p_max * r supported
int set_err(int code, const char *fmt, ...);
int cuda_err(cudaError_t e, const char *where);

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

struct pseudo_ctx {
    int dev = 0;
    int n = 0, n_pad = 0;
    double2 *U64 = nullptr, *L64 = nullptr;  // packed panels of T and T^H, FP64
    float2 *U32 = nullptr, *L32 = nullptr;   // the same in FP32
    double2 *diag = nullptr;                 // T_ii (the eigenvalues of C)
    double norm_fro = 0.0, norm2 = 0.0;      // ||T||_F and a 2-norm estimate
    pseudo_stats_t stats;
};

namespace pseudo {
void invlanc_carve(pseudo_ctx *h, const pseudo_opts *o, int64_t npts, Carver &c, void *plan);
int invlanc_run(pseudo_ctx *h, const pseudo_opts *o, const GridIO &io, Carver &c, cudaStream_t s);
void recycle_carve(pseudo_ctx *h, const pseudo_opts *o, int64_t npts, Carver &c, void *plan);
int recycle_run(pseudo_ctx *h, const pseudo_opts *o, const GridIO &io, Carver &c, cudaStream_t s);
void launch_convert_64_to_32(const double2 *a, float2 *b, int64_t cnt, cudaStream_t s);
void launch_convert_32_to_64(const float2 *a, double2 *b, int64_t cnt, cudaStream_t s);
}  // namespace pseudo
