// Many matrices of uneven size in one call (pseudo_grid_batch).
//
// Every matrix has its own Schur factor (handle) and its own grid.  The call
// runs the single-matrix driver for all of them concurrently: a pool of host
// workers, each with its own CUDA stream and its own slice of the caller's
// workspace, takes a fixed share of the matrices (largest first, balanced by
// work); kernels of different matrices overlap on the GPU, so small matrices
// that cannot fill 148 SMs alone fill them together.  The caller's stream is
// ordered before the first and after the last piece of work with events.
#include <algorithm>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "driver.h"
#include "internal.h"

using namespace pseudo;

namespace {
constexpr int BATCH_WORKERS = 8;

int slice_bytes(const pseudo_handle *hs, int nmat, const int64_t *npts, const pseudo_opts *o, size_t *out) {
    size_t mx = 0;
    for (int m = 0; m < nmat; ++m) {
        size_t b = 0;
        const int rc = pseudo_workspace_bytes(hs[m], o, npts[m], &b);
        if (rc) return rc;
        mx = std::max(mx, b);
    }
    *out = (mx + 255) & ~(size_t)255;
    return PSEUDO_OK;
}
}  // namespace

extern "C" int pseudo_grid_batch_workspace_bytes(const pseudo_handle *hs, int nmat, const int64_t *npts,
                                                 const pseudo_opts *o, size_t *bytes) {
    if (!hs || !npts || !o || !bytes || nmat < 1) return set_err(PSEUDO_ERR_ARG, "bad argument");
    size_t slice = 0;
    const int rc = slice_bytes(hs, nmat, npts, o, &slice);
    if (rc) return rc;
    *bytes = slice * (size_t)std::min(nmat, BATCH_WORKERS) + 256;
    return PSEUDO_OK;
}

extern "C" int pseudo_grid_batch(const pseudo_handle *hs, int nmat, const pseudo_c64 *const *z, const int64_t *npts,
                                 const double *eps_levels, int neps, const pseudo_opts *o, double *const *sigma_out,
                                 double *const *res_out, int32_t *const *flags_out, uint32_t *const *member_out,
                                 void *workspace, size_t workspace_bytes, void *stream) {
    if (!hs || !z || !npts || !o || !sigma_out || nmat < 1) return set_err(PSEUDO_ERR_ARG, "bad argument");
    for (int m = 0; m < nmat; ++m)
        if (!hs[m] || (npts[m] > 0 && (!z[m] || !sigma_out[m]))) return set_err(PSEUDO_ERR_ARG, "matrix %d: bad argument", m);
    for (int m = 0; m < nmat; ++m)
        for (int q = 0; q < m; ++q)
            if (hs[m] == hs[q]) return set_err(PSEUDO_ERR_ARG, "matrix %d repeats the handle of matrix %d", m, q);
    size_t slice = 0;
    int rc = slice_bytes(hs, nmat, npts, o, &slice);
    if (rc) return rc;
    const int nw = std::min(nmat, BATCH_WORKERS);
    if (!workspace || workspace_bytes < slice * nw + 256)
        return set_err(PSEUDO_ERR_WORKSPACE, "workspace needs %zu bytes", slice * nw + 256);
    char *base = (char *)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaStream_t caller = (cudaStream_t)stream;
    // the workers' streams and events; on a failure nothing has been launched
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t start = nullptr;
    auto release = [&]() {
        for (cudaEvent_t ev : done) cudaEventDestroy(ev);
        for (cudaStream_t st : streams) cudaStreamDestroy(st);
        if (start) cudaEventDestroy(start);
    };
    cudaError_t e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        start = nullptr;
        return cuda_err(e, "pseudo_grid_batch: event");
    }
    for (int w = 0; w < nw; ++w) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
            release();
            return cuda_err(e, "pseudo_grid_batch: stream");
        }
        streams.push_back(st);
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            release();
            return cuda_err(e, "pseudo_grid_batch: event");
        }
        done.push_back(ev);
    }
    if ((e = cudaEventRecord(start, caller)) != cudaSuccess) {
        release();
        return cuda_err(e, "pseudo_grid_batch: stream");
    }
    // Matrices go to workers by a fixed rule (largest first, each to the worker
    // with the least work so far, work ~ n^2 x points), so that a repeated call
    // puts every matrix on the same workspace slice and stream again -- the
    // handle's cached loop graph then matches.
    std::vector<int> order(nmat);
    std::iota(order.begin(), order.end(), 0);
    auto cost = [&](int m) { return (double)hs[m]->n * hs[m]->n * (double)npts[m]; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<std::vector<int>> assigned(nw);
    {
        std::vector<double> load(nw, 0.0);
        for (int m : order) {
            const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            assigned[w].push_back(m);
            load[w] += cost(m);
        }
    }
    // host-driven loops: replayed conditional-node graphs on the workers'
    // streams overlapped less on the device (64 Gaussian matrices, n 256..2048:
    // 171k points/s against 218k)
    pseudo_opts oh = *o;
    oh.device_loop = 0;
    std::vector<int> results(nmat, PSEUDO_OK);
    std::vector<std::string> errors(nmat);
    auto worker = [&](int w) {
        cudaSetDevice(dev);
        cudaStreamWaitEvent(streams[w], start, 0);
        for (const int m : assigned[w]) {
            if (npts[m] == 0) continue;
            const int r = pseudo_grid(hs[m], z[m], npts[m], eps_levels, neps, &oh, sigma_out[m],
                                      res_out ? res_out[m] : nullptr, flags_out ? flags_out[m] : nullptr,
                                      member_out ? member_out[m] : nullptr, base + (size_t)w * slice, slice,
                                      streams[w]);
            results[m] = r;
            if (r < 0) errors[m] = pseudo_last_error();
        }
        cudaEventRecord(done[w], streams[w]);
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < nw; ++w) pool.emplace_back(worker, w);
    for (auto &t : pool) t.join();
    for (int w = 0; w < nw; ++w) cudaStreamWaitEvent(caller, done[w], 0);
    release();
    rc = PSEUDO_OK;
    for (int m = 0; m < nmat; ++m) {
        if (results[m] < 0) return set_err(results[m], "matrix %d: %s", m, errors[m].c_str());
        if (results[m] > rc) rc = results[m];
    }
    return rc;
}
